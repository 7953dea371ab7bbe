// Hierarchy setup kernels: fine-level assembly, MIS-2 aggregation, multiplier aggregation
// (Algorithm 1), tentative transfers by per-aggregate QR, smoothed prolongator, block SpGEMM
// Galerkin products, CheapSIMPLE data and the coarsest dense inverse.
#include "amgc_internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

namespace amgc {

// ======================================================================== small utilities
__device__ __forceinline__ void set_status(int* st, int bit) { atomicOr(st, bit); }

__global__ void k_iota(int n, int* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = i;
}
__global__ void k_fill_int(int64_t n, int v, int* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = v;
}
__global__ void k_fill_dbl(int64_t n, double v, double* __restrict__ y) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = v;
}

// Sorts each segment [ptr[s], ptr[s+1]) of (key, payload) by key (insertion sort; segments are short).
__global__ void k_sort_segments(int nseg, const int* __restrict__ ptr, int* __restrict__ key, int* __restrict__ pay) {
  int sgi = blockIdx.x * blockDim.x + threadIdx.x;
  if (sgi >= nseg) return;
  int b = ptr[sgi], e = ptr[sgi + 1];
  for (int i = b + 1; i < e; ++i) {
    int k = key[i], p = pay ? pay[i] : 0;
    int j = i - 1;
    while (j >= b && key[j] > k) {
      key[j + 1] = key[j];
      if (pay) pay[j + 1] = pay[j];
      --j;
    }
    key[j + 1] = k;
    if (pay) pay[j + 1] = p;
  }
}

// Same, one warp per segment: each element's rank is the number of smaller keys (keys are
// distinct within a segment); segments longer than the shared buffer fall back to one thread.
constexpr int kSortCap = 1024;
constexpr int kSortWarps = 4;
__global__ void __launch_bounds__(kSortWarps * 32)
k_sort_segments_warp(int nseg, const int* __restrict__ ptr, int* __restrict__ key, int* __restrict__ pay) {
  __shared__ int sk[kSortWarps][kSortCap];
  __shared__ int sp[kSortWarps][kSortCap];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int sgi = blockIdx.x * kSortWarps + wid;
  if (sgi >= nseg) return;
  const int b = ptr[sgi], e = ptr[sgi + 1], n = e - b;
  if (n <= 1) return;
  if (n > kSortCap) {
    if (lane == 0) {
      for (int i = b + 1; i < e; ++i) {
        int k = key[i], p = pay ? pay[i] : 0;
        int j = i - 1;
        while (j >= b && key[j] > k) {
          key[j + 1] = key[j];
          if (pay) pay[j + 1] = pay[j];
          --j;
        }
        key[j + 1] = k;
        if (pay) pay[j + 1] = p;
      }
    }
    return;
  }
  for (int i = lane; i < n; i += 32) {
    sk[wid][i] = key[b + i];
    if (pay) sp[wid][i] = pay[b + i];
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const int k = sk[wid][i];
    int r = 0;
    for (int j = 0; j < n; ++j) r += sk[wid][j] < k;
    key[b + r] = k;
    if (pay) pay[b + r] = sp[wid][i];
  }
}

// Counting sort of items 0..n-1 by bucket id: out ptr (nb+1) and idx (items sorted by bucket,
// ascending item id inside a bucket).
__global__ void k_count(int n, const int* __restrict__ bucket, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && bucket[i] >= 0) atomicAdd(cnt + bucket[i], 1);
}
__global__ void k_scatter(int n, const int* __restrict__ bucket, int* __restrict__ cursor, int* __restrict__ idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && bucket[i] >= 0) idx[atomicAdd(cursor + bucket[i], 1)] = i;
}
__global__ void k_copy_int(int n, const int* __restrict__ a, int* __restrict__ b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

int bucket_lists(int n, const int* bucket, int nb, DBuf<int>& ptr, DBuf<int>& idx, cudaStream_t s) {
  AMGC_TRY(ptr.alloc(nb + 1));
  DBuf<int> cur;
  AMGC_TRY(cur.alloc(nb + 1));
  AMGC_CUDA_TRY(cudaMemsetAsync(ptr.p, 0, (nb + 1) * sizeof(int), s));
  if (n > 0) AMGC_LAUNCH(k_count<<<div_up(n, 256), 256, 0, s>>>(n, bucket, ptr.p));
  int total = 0;
  AMGC_TRY(exclusive_scan(ptr.p, ptr.p, nb + 1, s, &total));
  AMGC_TRY(idx.alloc(std::max(total, 1)));
  AMGC_LAUNCH(k_copy_int<<<div_up(nb + 1, 256), 256, 0, s>>>(nb + 1, ptr.p, cur.p));
  if (n > 0) AMGC_LAUNCH(k_scatter<<<div_up(n, 256), 256, 0, s>>>(n, bucket, cur.p, idx.p));
  if (nb > 0) AMGC_LAUNCH(k_sort_segments_warp<<<div_up(nb, kSortWarps), kSortWarps * 32, 0, s>>>(nb, ptr.p, idx.p, nullptr));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

int check_status(amgc_hierarchy* h, const char* where) {
  int st = 0;
  AMGC_CUDA_TRY(cudaMemcpyAsync(&st, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  AMGC_CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (st == 0) return AMGC_OK;
  AMGC_CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(int), h->stream));
  std::string m = std::string(where) + ":";
  if (st & ST_BAD_INDEX) m += " index out of range or unsorted;";
  if (st & ST_NO_DIAG) m += " missing diagonal block;";
  if (st & ST_SINGULAR) m += " singular block or pivot;";
  if (st & ST_RANK) m += " rank-deficient nullspace on an aggregate;";
  if (st & ST_ROW_TOO_DENSE) m += " product row exceeds the hash capacity;";
  if (st & ST_NONFINITE) m += " non-finite value;";
  if (st & ST_TIMEOUT) m += " a bounded wait on an asynchronous copy gave up;";
  set_error(m);
  if (st & ST_TIMEOUT) return AMGC_TIMEOUT;
  if (st & (ST_SINGULAR | ST_RANK)) return AMGC_ESINGULAR;
  return AMGC_EINVAL;
}

// ======================================================================== fine-level assembly
__global__ void k_validate_bsr(int nbr, int nbc, const int* __restrict__ rp, const int* __restrict__ col,
                               int require_diag, int* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  int b = rp[i], e = rp[i + 1];
  if (e < b) { set_status(st, ST_BAD_INDEX); return; }
  bool diag = false;
  for (int q = b; q < e; ++q) {
    int c = col[q];
    if (c < 0 || c >= nbc || (q > b && col[q - 1] >= c)) set_status(st, ST_BAD_INDEX);
    if (c == i) diag = true;
  }
  if (require_diag && !diag) set_status(st, ST_NO_DIAG);
}
__global__ void k_validate_index(int n, const int* __restrict__ a, int hi, int* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (a[i] < 0 || a[i] >= hi)) set_status(st, ST_BAD_INDEX);
}
__global__ void k_role(int n, const int* __restrict__ node, int* __restrict__ role, int* st) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (atomicCAS(role + node[j], -1, j) != -1) set_status(st, ST_BAD_INDEX);   // duplicate node
}
__global__ void k_role_clash(int n, const int* __restrict__ a, const int* __restrict__ b, int* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && a[i] >= 0 && b[i] >= 0) set_status(st, ST_BAD_INDEX);
}
__global__ void k_b1_count(int nn, const int* __restrict__ sl_of, const int* __restrict__ ms_of,
                           const int* __restrict__ mt_ptr, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int c = 0;
  if (sl_of[i] >= 0) c += 1;
  if (ms_of[i] >= 0) c += mt_ptr[ms_of[i] + 1] - mt_ptr[ms_of[i]];
  cnt[i] = c;
}
// B1 row i: slave node -> (j, D_j I3); master node l -> (j, -M_jl I3) for the sorted slaves j of column l.
__global__ void k_b1_fill(int nn, const int* __restrict__ rp, const int* __restrict__ sl_of, const int* __restrict__ ms_of,
                          const double* __restrict__ D, const int* __restrict__ mt_ptr, const int* __restrict__ mt_idx,
                          const int* __restrict__ m_pos, const double* __restrict__ Mval, int* __restrict__ col,
                          double* __restrict__ val) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int q = rp[i];
  auto put = [&](int j, double a) {
    col[q] = j;
    double* v = val + (int64_t)q * 9;
    for (int t = 0; t < 9; ++t) v[t] = 0.0;
    v[0] = v[4] = v[8] = a;
    ++q;
  };
  if (sl_of[i] >= 0) put(sl_of[i], D[sl_of[i]]);
  if (ms_of[i] >= 0) {
    int l = ms_of[i];
    for (int e = mt_ptr[l]; e < mt_ptr[l + 1]; ++e) put(mt_idx[e], -Mval[m_pos[e]]);
  }
}
// M^T: per master column, the slave rows (mt_idx) and the positions in M's value array (m_pos)
__global__ void k_mt_count(int ns, const int* __restrict__ mrp, const int* __restrict__ mcol, int nm,
                           int* __restrict__ cnt, int* st) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ns) return;
  for (int q = mrp[j]; q < mrp[j + 1]; ++q) {
    int l = mcol[q];
    if (l < 0 || l >= nm) { set_status(st, ST_BAD_INDEX); continue; }
    atomicAdd(cnt + l, 1);
  }
}
__global__ void k_mt_scatter(int ns, const int* __restrict__ mrp, const int* __restrict__ mcol, int nm,
                             int* __restrict__ cur, int* __restrict__ mt_idx, int* __restrict__ m_pos) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ns) return;
  for (int q = mrp[j]; q < mrp[j + 1]; ++q) {
    int l = mcol[q];
    if (l < 0 || l >= nm) continue;
    int p = atomicAdd(cur + l, 1);
    mt_idx[p] = j;
    m_pos[p] = q;
  }
}
__global__ void k_b2_count(int ns, const uint8_t* __restrict__ active, const int* __restrict__ mrp, int* __restrict__ cnt) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ns) cnt[j] = active[j] ? 1 + (mrp[j + 1] - mrp[j]) : 0;
}
// B2 row j (active): n^T on the slave node (times D_j) and on the master nodes (times -M_jl),
// sorted by node; Z block: active (0; -tau_xi; -tau_eta), inactive -I3.
__global__ void k_b2_fill(int ns, const uint8_t* __restrict__ active, const int* __restrict__ rp,
                          const int* __restrict__ slave_node, const int* __restrict__ master_node,
                          const double* __restrict__ D, const int* __restrict__ mrp, const int* __restrict__ mcol,
                          const double* __restrict__ mval, const double* __restrict__ triad, int* __restrict__ col,
                          double* __restrict__ val, double* __restrict__ Z) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ns) return;
  const double* T = triad + (int64_t)j * 9;
  double* z = Z + (int64_t)j * 9;
  if (!active[j]) {
    for (int t = 0; t < 9; ++t) z[t] = 0.0;
    z[0] = z[4] = z[8] = -1.0;
    return;
  }
  z[0] = z[1] = z[2] = 0.0;
  for (int t = 0; t < 3; ++t) {
    z[3 + t] = -T[3 + t];
    z[6 + t] = -T[6 + t];
  }
  int b = rp[j];
  int q = b;
  auto put = [&](int node, double a) {
    // insertion into the sorted row
    int p = q;
    while (p > b && col[p - 1] > node) {
      col[p] = col[p - 1];
      for (int t = 0; t < 9; ++t) val[(int64_t)p * 9 + t] = val[(int64_t)(p - 1) * 9 + t];
      --p;
    }
    col[p] = node;
    double* v = val + (int64_t)p * 9;
    v[0] = a * T[0];
    v[1] = a * T[1];
    v[2] = a * T[2];
    for (int t = 3; t < 9; ++t) v[t] = 0.0;
    ++q;
  };
  put(slave_node[j], D[j]);
  for (int e = mrp[j]; e < mrp[j + 1]; ++e) put(master_node[mcol[e]], -mval[e]);
}

int build_fine_level(amgc_hierarchy* h, const amgc_bsr* K, const double* D, const amgc_csr* M,
                     const int* slave_node, const int* master_node, const double* triad,
                     const uint8_t* active, const int* body_id, const double* nullspace) {
  cudaStream_t s = h->stream;
  Level& L = h->L[0];
  const int nn = K->n_brow, ns = M->n_row, nm = M->n_col;
  L.nn = nn;
  L.bu = 3;
  L.nl = ns;
  // --- K
  int kn = 0;
  AMGC_CUDA_TRY(cudaMemcpy(&kn, K->rowptr + nn, sizeof(int), cudaMemcpyDefault));
  L.K.nbr = nn; L.K.nbc = nn; L.K.br = 3; L.K.bc = 3; L.K.nnzb = kn;
  AMGC_TRY(L.K.rowptr.alloc(nn + 1));
  AMGC_TRY(L.K.col.alloc(std::max(kn, 1)));
  AMGC_TRY(L.K.val.alloc((size_t)std::max(kn, 1) * 9));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.K.rowptr.p, K->rowptr, (nn + 1) * sizeof(int), cudaMemcpyDefault, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.K.col.p, K->col, (size_t)kn * sizeof(int), cudaMemcpyDefault, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.K.val.p, K->val, (size_t)kn * 9 * sizeof(double), cudaMemcpyDefault, s));
  AMGC_LAUNCH(k_validate_bsr<<<div_up(nn, 256), 256, 0, s>>>(nn, nn, L.K.rowptr.p, L.K.col.p, 1, h->status.p));
  AMGC_TRY(check_status(h, "K"));
  // --- per-node arrays
  AMGC_TRY(L.body.alloc(nn));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.body.p, body_id, nn * sizeof(int), cudaMemcpyDefault, s));
  AMGC_TRY(L.B.alloc((size_t)nn * 3 * 6));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.B.p, nullspace, (size_t)nn * 18 * sizeof(double), cudaMemcpyDefault, s));
  // --- interface data
  DBuf<double> dD, dMv, dT;
  DBuf<int> dMrp, dMcol, dSl, dMs;
  DBuf<uint8_t> dAct;
  int mnnz = 0;
  AMGC_CUDA_TRY(cudaMemcpy(&mnnz, M->rowptr + ns, sizeof(int), cudaMemcpyDefault));
  AMGC_TRY(dD.alloc(std::max(ns, 1)));
  AMGC_TRY(dMv.alloc(std::max(mnnz, 1)));
  AMGC_TRY(dT.alloc((size_t)std::max(ns, 1) * 9));
  AMGC_TRY(dMrp.alloc(ns + 1));
  AMGC_TRY(dMcol.alloc(std::max(mnnz, 1)));
  AMGC_TRY(dSl.alloc(std::max(ns, 1)));
  AMGC_TRY(dMs.alloc(std::max(nm, 1)));
  AMGC_TRY(dAct.alloc(std::max(ns, 1)));
  if (ns > 0) {
    AMGC_CUDA_TRY(cudaMemcpyAsync(dD.p, D, ns * sizeof(double), cudaMemcpyDefault, s));
    AMGC_CUDA_TRY(cudaMemcpyAsync(dT.p, triad, (size_t)ns * 9 * sizeof(double), cudaMemcpyDefault, s));
    AMGC_CUDA_TRY(cudaMemcpyAsync(dSl.p, slave_node, ns * sizeof(int), cudaMemcpyDefault, s));
    AMGC_CUDA_TRY(cudaMemcpyAsync(dAct.p, active, ns, cudaMemcpyDefault, s));
  }
  AMGC_CUDA_TRY(cudaMemcpyAsync(dMrp.p, M->rowptr, (ns + 1) * sizeof(int), cudaMemcpyDefault, s));
  if (mnnz > 0) {
    AMGC_CUDA_TRY(cudaMemcpyAsync(dMv.p, M->val, (size_t)mnnz * sizeof(double), cudaMemcpyDefault, s));
    AMGC_CUDA_TRY(cudaMemcpyAsync(dMcol.p, M->col, (size_t)mnnz * sizeof(int), cudaMemcpyDefault, s));
  }
  if (nm > 0) AMGC_CUDA_TRY(cudaMemcpyAsync(dMs.p, master_node, nm * sizeof(int), cudaMemcpyDefault, s));
  if (ns > 0) AMGC_LAUNCH(k_validate_index<<<div_up(ns, 256), 256, 0, s>>>(ns, dSl.p, nn, h->status.p));
  if (nm > 0) AMGC_LAUNCH(k_validate_index<<<div_up(nm, 256), 256, 0, s>>>(nm, dMs.p, nn, h->status.p));
  AMGC_TRY(check_status(h, "interface node ids"));
  // roles of the displacement nodes
  DBuf<int> sl_of, ms_of;
  AMGC_TRY(sl_of.alloc(nn));
  AMGC_TRY(ms_of.alloc(nn));
  AMGC_LAUNCH(k_fill_int<<<div_up(nn, 256), 256, 0, s>>>(nn, -1, sl_of.p));
  AMGC_LAUNCH(k_fill_int<<<div_up(nn, 256), 256, 0, s>>>(nn, -1, ms_of.p));
  if (ns > 0) AMGC_LAUNCH(k_role<<<div_up(ns, 256), 256, 0, s>>>(ns, dSl.p, sl_of.p, h->status.p));
  if (nm > 0) AMGC_LAUNCH(k_role<<<div_up(nm, 256), 256, 0, s>>>(nm, dMs.p, ms_of.p, h->status.p));
  AMGC_LAUNCH(k_role_clash<<<div_up(nn, 256), 256, 0, s>>>(nn, sl_of.p, ms_of.p, h->status.p));
  // M^T
  DBuf<int> mt_ptr, mt_cur, mt_idx, m_pos;
  AMGC_TRY(mt_ptr.alloc(nm + 1));
  AMGC_TRY(mt_cur.alloc(nm + 1));
  AMGC_TRY(mt_idx.alloc(std::max(mnnz, 1)));
  AMGC_TRY(m_pos.alloc(std::max(mnnz, 1)));
  AMGC_CUDA_TRY(cudaMemsetAsync(mt_ptr.p, 0, (nm + 1) * sizeof(int), s));
  if (ns > 0) AMGC_LAUNCH(k_mt_count<<<div_up(ns, 256), 256, 0, s>>>(ns, dMrp.p, dMcol.p, nm, mt_ptr.p, h->status.p));
  AMGC_TRY(check_status(h, "mortar M"));
  AMGC_TRY(exclusive_scan(mt_ptr.p, mt_ptr.p, nm + 1, s, nullptr));
  AMGC_LAUNCH(k_copy_int<<<div_up(nm + 1, 256), 256, 0, s>>>(nm + 1, mt_ptr.p, mt_cur.p));
  if (ns > 0) AMGC_LAUNCH(k_mt_scatter<<<div_up(ns, 256), 256, 0, s>>>(ns, dMrp.p, dMcol.p, nm, mt_cur.p, mt_idx.p, m_pos.p));
  if (nm > 0) AMGC_LAUNCH(k_sort_segments_warp<<<div_up(nm, kSortWarps), kSortWarps * 32, 0, s>>>(nm, mt_ptr.p, mt_idx.p, m_pos.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  // --- B1 (nn x ns, 3x3)
  L.B1.nbr = nn; L.B1.nbc = ns; L.B1.br = 3; L.B1.bc = 3;
  AMGC_TRY(L.B1.rowptr.alloc(nn + 1));
  AMGC_CUDA_TRY(cudaMemsetAsync(L.B1.rowptr.p, 0, (nn + 1) * sizeof(int), s));   // entry nn joins the scan
  AMGC_LAUNCH(k_b1_count<<<div_up(nn, 256), 256, 0, s>>>(nn, sl_of.p, ms_of.p, mt_ptr.p, L.B1.rowptr.p));
  int b1n = 0;
  AMGC_TRY(exclusive_scan(L.B1.rowptr.p, L.B1.rowptr.p, nn + 1, s, &b1n));
  L.B1.nnzb = b1n;
  AMGC_TRY(L.B1.col.alloc(std::max(b1n, 1)));
  AMGC_TRY(L.B1.val.alloc((size_t)std::max(b1n, 1) * 9));
  AMGC_LAUNCH(k_b1_fill<<<div_up(nn, 256), 256, 0, s>>>(nn, L.B1.rowptr.p, sl_of.p, ms_of.p, dD.p, mt_ptr.p, mt_idx.p, m_pos.p,
                                            dMv.p, L.B1.col.p, L.B1.val.p));
  // --- B2 (ns x nn, 3x3) and Z
  L.B2.nbr = ns; L.B2.nbc = nn; L.B2.br = 3; L.B2.bc = 3;
  AMGC_TRY(L.B2.rowptr.alloc(ns + 1));
  AMGC_CUDA_TRY(cudaMemsetAsync(L.B2.rowptr.p, 0, (ns + 1) * sizeof(int), s));   // entry ns joins the scan
  if (ns > 0) AMGC_LAUNCH(k_b2_count<<<div_up(ns, 256), 256, 0, s>>>(ns, dAct.p, dMrp.p, L.B2.rowptr.p));
  int b2n = 0;
  AMGC_TRY(exclusive_scan(L.B2.rowptr.p, L.B2.rowptr.p, ns + 1, s, &b2n));
  L.B2.nnzb = b2n;
  AMGC_TRY(L.B2.col.alloc(std::max(b2n, 1)));
  AMGC_TRY(L.B2.val.alloc((size_t)std::max(b2n, 1) * 9));
  AMGC_TRY(L.Z.alloc((size_t)std::max(ns, 1) * 9));
  if (ns > 0)
    AMGC_LAUNCH(k_b2_fill<<<div_up(ns, 256), 256, 0, s>>>(ns, dAct.p, L.B2.rowptr.p, dSl.p, dMs.p, dD.p, dMrp.p, dMcol.p, dMv.p,
                                              dT.p, L.B2.col.p, L.B2.val.p, L.Z.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(check_status(h, "interface assembly"));
  // --- interface data kept for active-set updates
  L.if_D = std::move(dD);
  L.if_Mv = std::move(dMv);
  L.if_T = std::move(dT);
  L.if_Mrp = std::move(dMrp);
  L.if_Mcol = std::move(dMcol);
  L.if_Sl = std::move(dSl);
  L.if_Ms = std::move(dMs);
  L.if_act = std::move(dAct);
  // --- multiplier data
  AMGC_TRY(L.Bl.alloc(std::max(ns, 1)));
  AMGC_LAUNCH(k_fill_dbl<<<div_up(std::max(ns, 1), 256), 256, 0, s>>>(ns, 1.0, L.Bl.p));
  AMGC_TRY(L.lm_dnode.alloc(std::max(ns, 1)));
  if (ns > 0) AMGC_LAUNCH(k_copy_int<<<div_up(ns, 256), 256, 0, s>>>(ns, L.if_Sl.p, L.lm_dnode.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

// ======================================================================== MIS-2 aggregation
// Priority of node i: fmix32(i ^ seed) * 2^32 + i (fmix32 in amgc_internal.cuh); the stored
// value is priority + 1 for an undecided node and 0 otherwise.
enum : int8_t { UND = 0, ROOT = 1, OUT = 2 };

// key_base (batched hierarchies): first node of the node's instance, so that the hash uses the
// instance-local index and every instance aggregates exactly as it would alone
__global__ void k_mis_key(int n, const int8_t* __restrict__ state, uint32_t seed, const int* __restrict__ key_base,
                          unsigned long long* __restrict__ kv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t li = (uint32_t)(key_base ? i - key_base[i] : i);
  unsigned long long key = ((unsigned long long)fmix32(li ^ seed) << 32) | (unsigned long long)(uint32_t)i;
  kv[i] = state[i] == UND ? key + 1ull : 0ull;
}
// out[i] = max(in[i], max over graph neighbours j of in[j]); the graph is K's pattern without
// the diagonal and without couplings between different bodies.
__global__ void k_mis_max(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ body,
                          const unsigned long long* __restrict__ in, unsigned long long* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = in[i];
  const int bi = body[i];
  for (int q = rp[i]; q < rp[i + 1]; ++q) {
    int j = col[q];
    if (j == i || body[j] != bi) continue;
    unsigned long long v = in[j];
    m = v > m ? v : m;
  }
  out[i] = m;
}
__global__ void k_mis_newroot(int n, const unsigned long long* __restrict__ kv, const unsigned long long* __restrict__ m2,
                              int8_t* __restrict__ state, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = (state[i] == UND && kv[i] == m2[i]) ? 1 : 0;
  flag[i] = f;
}
__global__ void k_mis_any(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ body,
                          const int* __restrict__ in, int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = in[i];
  const int bi = body[i];
  for (int q = rp[i]; q < rp[i + 1] && !a; ++q) {
    int j = col[q];
    if (j == i || body[j] != bi) continue;
    a |= in[j];
  }
  out[i] = a;
}
__global__ void k_mis_mark(int n, const int* __restrict__ newroot, const int* __restrict__ near2, int8_t* __restrict__ state,
                           int* __restrict__ undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int8_t st = state[i];
  if (st == UND) {
    if (newroot[i]) st = ROOT;
    else if (near2[i]) st = OUT;
    state[i] = st;
  }
  if (st == UND) atomicAdd(undecided, 1);
}
__global__ void k_root_flag(int n, const int8_t* __restrict__ state, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == ROOT ? 1 : 0;
}
// phase 1/2: root -> own aggregate; neighbour of a root -> the root's aggregate
__global__ void k_agg_phase2(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ body,
                             const int8_t* __restrict__ state, const int* __restrict__ rank, int* __restrict__ agg,
                             int* __restrict__ roots) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (state[i] == ROOT) {
    agg[i] = rank[i];
    roots[rank[i]] = i;
    return;
  }
  int a = -1;
  const int bi = body[i];
  for (int q = rp[i]; q < rp[i + 1]; ++q) {
    int j = col[q];
    if (j == i || body[j] != bi) continue;
    if (state[j] == ROOT) { a = rank[j]; break; }
  }
  agg[i] = a;
}
// phase 3: unassigned node -> phase-2 aggregate with most shared edges, ties to the smallest id.
// One warp per node: each lane scores the candidates of its share of the neighbours (every
// neighbour is counted for every candidate), then the warp keeps the best (count, id) pair.
__global__ void k_agg_phase3(int n, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ body,
                             const int* __restrict__ agg2, int* __restrict__ agg, int* st) {
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= n) return;
  const int own = agg2[i];
  if (own >= 0) {
    if (lane == 0) agg[i] = own;
    return;
  }
  const int bi = body[i];
  int best = -1, best_cnt = 0;
  const int b = rp[i], e = rp[i + 1];
  for (int q = b + lane; q < e; q += 32) {
    int j = col[q];
    if (j == i || body[j] != bi) continue;
    int a = agg2[j];
    if (a < 0) continue;
    int cnt = 0;
    for (int r = b; r < e; ++r) {
      int k = col[r];
      if (k == i || body[k] != bi) continue;
      cnt += agg2[k] == a;
    }
    if (cnt > best_cnt || (cnt == best_cnt && a < best)) { best = a; best_cnt = cnt; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int oc = __shfl_xor_sync(0xffffffffu, best_cnt, o);
    const int oa = __shfl_xor_sync(0xffffffffu, best, o);
    if (oc > best_cnt || (oc == best_cnt && oa >= 0 && (best < 0 || oa < best))) { best = oa; best_cnt = oc; }
  }
  if (lane == 0) {
    if (best < 0) set_status(st, ST_BAD_INDEX);
    agg[i] = best;
  }
}

static int mis2_aggregate(amgc_hierarchy* h, Level& L, DBuf<int>& roots, int* n_agg) {
  cudaStream_t s = h->stream;
  const int n = L.nn;
  DBuf<int8_t> state;
  DBuf<unsigned long long> kv, m1, m2;
  DBuf<int> nr, a1, a2, cnt;
  AMGC_TRY(state.alloc(n));
  AMGC_TRY(kv.alloc(n));
  AMGC_TRY(m1.alloc(n));
  AMGC_TRY(m2.alloc(n));
  AMGC_TRY(nr.alloc(n + 1));
  AMGC_TRY(a1.alloc(n));
  AMGC_TRY(a2.alloc(n));
  AMGC_TRY(cnt.alloc(1));
  AMGC_CUDA_TRY(cudaMemsetAsync(state.p, 0, n, s));
  const int g = div_up(n, 256);
  const int* rp = L.K.rowptr.p;
  const int* col = L.K.col.p;
  const int* body = L.body.p;
  for (int round = 0; round < 10000; ++round) {
    AMGC_LAUNCH(k_mis_key<<<g, 256, 0, s>>>(n, state.p, h->opts.seed, L.key_base.p, kv.p));
    AMGC_LAUNCH(k_mis_max<<<g, 256, 0, s>>>(n, rp, col, body, kv.p, m1.p));
    AMGC_LAUNCH(k_mis_max<<<g, 256, 0, s>>>(n, rp, col, body, m1.p, m2.p));
    AMGC_LAUNCH(k_mis_newroot<<<g, 256, 0, s>>>(n, kv.p, m2.p, state.p, nr.p));
    AMGC_LAUNCH(k_mis_any<<<g, 256, 0, s>>>(n, rp, col, body, nr.p, a1.p));
    AMGC_LAUNCH(k_mis_any<<<g, 256, 0, s>>>(n, rp, col, body, a1.p, a2.p));
    AMGC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int), s));
    AMGC_LAUNCH(k_mis_mark<<<g, 256, 0, s>>>(n, nr.p, a2.p, state.p, cnt.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    int und = 0;
    AMGC_CUDA_TRY(cudaMemcpyAsync(&und, cnt.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
    if (und == 0) break;
  }
  // aggregate ids by ascending root id
  AMGC_LAUNCH(k_root_flag<<<g, 256, 0, s>>>(n, state.p, nr.p));
  int na = 0;
  AMGC_TRY(exclusive_scan(nr.p, nr.p, n, s, &na));
  if (na == 0) {
    set_error("aggregation produced no aggregate");
    return AMGC_EINVAL;
  }
  AMGC_TRY(roots.alloc(na));
  AMGC_LAUNCH(k_agg_phase2<<<g, 256, 0, s>>>(n, rp, col, body, state.p, nr.p, a1.p, roots.p));
  AMGC_TRY(L.agg.alloc(n));
  AMGC_LAUNCH(k_agg_phase3<<<div_up((int64_t)n * 32, 256), 256, 0, s>>>(n, rp, col, body, a1.p, L.agg.p, h->status.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(check_status(h, "aggregation"));
  *n_agg = na;
  return AMGC_OK;
}

// ======================================================================== multiplier aggregation (Algorithm 1)
// Scanning the slave displacement DOFs in increasing order, the multiplier aggregate of a
// displacement aggregate k is opened at the first slave DOF of k; since D couples each
// multiplier node to exactly one displacement node, aggregate k's multiplier aggregate is
// numbered by the rank of the smallest coupled displacement node of k.
__global__ void k_lm_first(int nl, const int* __restrict__ lm_dnode, const int* __restrict__ agg, int* __restrict__ first) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  int d = lm_dnode[l];
  atomicMin(first + agg[d], d);
}
__global__ void k_lm_mark(int nn, const int* __restrict__ agg, const int* __restrict__ first, int* __restrict__ mark) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn) mark[i] = first[agg[i]] == i ? 1 : 0;
}
__global__ void k_lm_assign(int nl, const int* __restrict__ lm_dnode, const int* __restrict__ agg, const int* __restrict__ first,
                            const int* __restrict__ rank, int* __restrict__ lagg, int* __restrict__ lm_dnode_c) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  int k = agg[lm_dnode[l]];
  int L = rank[first[k]];
  lagg[l] = L;
  lm_dnode_c[L] = k;    // all members of L map to the same k
}

// ======================================================================== tentative prolongator by QR
// One warp per aggregate, Cholesky QR applied twice (CholQR2) to the aggregate's nullspace rows
// (member nodes ascending, DOF-minor): each pass forms the 6 x 6 Gram matrix of the current
// rows (lanes over rows, then a warp sum: every lane ends with the same bits), its Cholesky
// factor R_p (positive diagonal) redundantly in every lane, and the rows times R_p^-1.  Two
// passes give orthonormal columns to rounding level for nullspaces far from rank deficiency,
// in four sweeps over the rows instead of a sequential Gram-Schmidt chain; the product R_2 R_1
// (positive diagonal) goes to the coarse nullspace and the rows to P-hat's blocks.  The rank
// test reads R_1's diagonal (min / max below 1e-12, or a non-positive pivot).
__device__ __forceinline__ int64_t qr_row_addr(const int* __restrict__ midx, int m0, int bu, int t) {
  const int node = midx[m0 + t / bu];
  return ((int64_t)node * bu + (t % bu)) * 6;
}
// one CholQR pass: rows of src (or of dst after the first pass) become rows of dst = src R^-1
// (src and dst may be the same array: each lane reads and writes only its own rows)
__device__ bool cholqr_pass(const int* __restrict__ midx, int m0, int bu, int nrows, const double* src, double* dst,
                            int lane, double (&R)[6][6]) {
  double g[21];
#pragma unroll
  for (int q = 0; q < 21; ++q) g[q] = 0.0;
  for (int t = lane; t < nrows; t += 32) {
    const double* b = src + qr_row_addr(midx, m0, bu, t);
    double v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = b[c];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i; j < 6; ++j) {
        const int q = i * 6 - (i * (i - 1)) / 2 + (j - i);   // packed upper triangle, row-major
        g[q] = fma(v[i], v[j], g[q]);
      }
  }
#pragma unroll
  for (int q = 0; q < 21; ++q) g[q] = warp_sum(g[q]);
  // Cholesky G = R^T R
  bool ok = true;
  {
    double G[6][6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i; j < 6; ++j) G[i][j] = g[i * 6 - (i * (i - 1)) / 2 + (j - i)];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
      for (int j = 0; j < 6; ++j) R[i][j] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double d = G[i][i];
#pragma unroll
      for (int k = 0; k < i; ++k) d = fma(-R[k][i], R[k][i], d);
      if (!(d > 0.0) || !isfinite(d)) { ok = false; d = 1.0; }
      const double rii = sqrt(d);
      R[i][i] = rii;
      const double inv = 1.0 / rii;
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        double e = G[i][j];
#pragma unroll
        for (int k = 0; k < i; ++k) e = fma(-R[k][i], R[k][j], e);
        R[i][j] = e * inv;
      }
    }
  }
  // Rinv, upper triangular: column j from R Rinv(:, j) = e_j by back substitution
  double Ri[6][6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
#pragma unroll
    for (int i = 5; i >= 0; --i) {
      double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = i + 1; k < 6; ++k) t = fma(-R[i][k], Ri[k][j], t);
      Ri[i][j] = i > j ? 0.0 : t / R[i][i];
    }
  }
  for (int t = lane; t < nrows; t += 32) {
    const int64_t o = qr_row_addr(midx, m0, bu, t);
    double v[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = src[o + c];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double y = 0.0;
#pragma unroll
      for (int i = 0; i <= j; ++i) y = fma(v[i], Ri[i][j], y);
      dst[o + j] = y;
    }
  }
  __syncwarp();
  return ok;
}
__global__ void k_tentative_qr(int n_agg, int bu, const int* __restrict__ mptr, const int* __restrict__ midx,
                               const double* __restrict__ B, double* __restrict__ Pval, double* __restrict__ Bc, int* st) {
  const int lane = threadIdx.x & 31;
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (a >= n_agg) return;
  const int m0 = mptr[a], m1 = mptr[a + 1];
  const int nrows = (m1 - m0) * bu;
  double R1[6][6], R2[6][6];
  const bool ok1 = cholqr_pass(midx, m0, bu, nrows, B, Pval, lane, R1);
  const bool ok2 = cholqr_pass(midx, m0, bu, nrows, Pval, Pval, lane, R2);
  double rmin = R1[0][0], rmax = R1[0][0];
#pragma unroll
  for (int c = 1; c < 6; ++c) {
    rmin = fmin(rmin, R1[c][c]);
    rmax = fmax(rmax, R1[c][c]);
  }
  if (nrows < 6 || !ok1 || !ok2 || !(rmin > 1e-12 * rmax)) {
    if (lane == 0) set_status(st, ST_RANK);
  }
  // R = R2 R1 (upper triangular), lane i < 6 writes row i
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (lane == i) {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double r = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) r = (k >= i && k <= j) ? fma(R2[i][k], R1[k][j], r) : r;
        Bc[((int64_t)a * 6 + i) * 6 + j] = r;
      }
    }
  }
}
__global__ void k_tentative_pattern(int nn, const int* __restrict__ agg, int* __restrict__ rp, int* __restrict__ col) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nn) {
    rp[i] = i;
    col[i] = agg[i];
  }
  if (i == nn) rp[nn] = nn;
}

// multiplier tentative transfer: norms per aggregate (members ascending), weights per node
__global__ void k_lm_norm(int nlc, const int* __restrict__ ptr, const int* __restrict__ idx, const double* __restrict__ Bl,
                          double* __restrict__ norm) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlc) return;
  double s = 0.0;
  for (int e = ptr[L]; e < ptr[L + 1]; ++e) {
    double v = Bl[idx[e]];
    s += v * v;
  }
  norm[L] = sqrt(s);
}
__global__ void k_lm_weight(int nl, const int* __restrict__ lagg, const double* __restrict__ Bl, const double* __restrict__ norm,
                            double* __restrict__ w) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < nl) w[l] = Bl[l] / norm[lagg[l]];
}
// P-hat^lambda as BSR (one block w_l I3 per row) and its transpose
__global__ void k_pl_bsr(int nl, const int* __restrict__ lagg, const double* __restrict__ w, int* __restrict__ rp,
                         int* __restrict__ col, double* __restrict__ val) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < nl) {
    rp[l] = l;
    col[l] = lagg[l];
    double* v = val + (int64_t)l * 9;
    for (int t = 0; t < 9; ++t) v[t] = 0.0;
    v[0] = v[4] = v[8] = w[l];
  }
  if (l == nl) rp[nl] = nl;
}
__global__ void k_rl_bsr(int nlc, const int* __restrict__ ptr, const int* __restrict__ idx, const double* __restrict__ w,
                         int* __restrict__ rp, int* __restrict__ col, double* __restrict__ val) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L < nlc) {
    rp[L] = ptr[L];
    for (int e = ptr[L]; e < ptr[L + 1]; ++e) {
      int l = idx[e];
      col[e] = l;
      double* v = val + (int64_t)e * 9;
      for (int t = 0; t < 9; ++t) v[t] = 0.0;
      v[0] = v[4] = v[8] = w[l];
    }
  }
  if (L == nlc) rp[nlc] = ptr[nlc];
}
// Z_c[L] = sum_{l in L} w_l^2 Z_l
__global__ void k_zc(int nlc, const int* __restrict__ ptr, const int* __restrict__ idx, const double* __restrict__ w,
                     const double* __restrict__ Z, double* __restrict__ Zc) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlc) return;
  double acc[9];
  for (int t = 0; t < 9; ++t) acc[t] = 0.0;
  for (int e = ptr[L]; e < ptr[L + 1]; ++e) {
    int l = idx[e];
    double w2 = w[l] * w[l];
    for (int t = 0; t < 9; ++t) acc[t] += w2 * Z[(int64_t)l * 9 + t];
  }
  for (int t = 0; t < 9; ++t) Zc[(int64_t)L * 9 + t] = acc[t];
}

// ======================================================================== block SpGEMM C = A B
// One warp per row of A with a shared-memory hash set of block columns (symbolic), then a
// numeric pass that walks A's row in order and lets the lanes take B's entries: within one
// A entry the lanes hit distinct C blocks, so no atomics are needed and the summation order
// is fixed (deterministic results).
constexpr int kHashCap = 1024;
constexpr int kGemmWarps = 4;

__device__ __forceinline__ int hash_insert(int* tab, int cap, int key) {
  unsigned slot = ((unsigned)key * 2654435761u) & (unsigned)(cap - 1);
  for (int probe = 0; probe < cap; ++probe) {
    int prev = atomicCAS(tab + slot, -1, key);
    if (prev == -1) return 1;
    if (prev == key) return 0;
    slot = (slot + 1) & (unsigned)(cap - 1);
  }
  return -1;
}

// MODE 0: count unique columns per row into cnt; MODE 1: write sorted unique columns into ccol.
// One warp per C row with an open-addressing table in shared memory, sized per row: a power of
// two of at least twice the row's candidate count (the sum of the B row lengths its A entries
// reach; at most kHashCap), so that clearing and compacting the table cost what the row needs.
// The lanes take lpe lanes per A entry (32 / lpe A entries at once), each lane a strided part
// of its B row.
template <int MODE>
__global__ void __launch_bounds__(kGemmWarps * 32)
k_spgemm_symbolic(int nrow, int lpe, const int* __restrict__ arp, const int* __restrict__ acol, const int* __restrict__ brp,
                  const int* __restrict__ bcol, int* __restrict__ cnt, const int* __restrict__ crp,
                  int* __restrict__ ccol, int* st) {
  __shared__ int tab[kGemmWarps][kHashCap];
  __shared__ int nlist[kGemmWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row = blockIdx.x * kGemmWarps + wid;
  if (row >= nrow) return;
  const int a0 = arp[row], a1 = arp[row + 1];
  int bound = 0;
  for (int e = a0 + lane; e < a1; e += 32) {
    const int k = acol[e];
    bound += brp[k + 1] - brp[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(0xffffffffu, bound, o);
  int cap = 64;
  while (cap < kHashCap && cap < 2 * bound) cap <<= 1;
  int* T = tab[wid];
  for (int k = lane; k < cap; k += 32) T[k] = -1;
  __syncwarp();
  int mine = 0;
  bool overflow = false;
  const int per = 32 / lpe;   // A entries per pass
  const int sub = lane % lpe;
  for (int e0 = a0; e0 < a1; e0 += per) {
    const int e = e0 + lane / lpe;
    if (e < a1) {
      const int k = acol[e];
      for (int t = brp[k] + sub; t < brp[k + 1]; t += lpe) {
        const int r = hash_insert(T, cap, bcol[t]);
        if (r < 0) overflow = true;
        else mine += r;
      }
    }
  }
  __syncwarp();
  int total = mine;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if (__any_sync(0xffffffffu, overflow) || total > (kHashCap * 3) / 4) {
    if (lane == 0) set_status(st, ST_ROW_TOO_DENSE);
    if (MODE == 0 && lane == 0) cnt[row] = 0;
    return;
  }
  if (MODE == 0) {
    if (lane == 0) cnt[row] = total;
    return;
  }
  // compact the keys in place (a key moves to a slot at or below its own, already read), then
  // rank them
  int* Ls = T;
  if (lane == 0) nlist[wid] = 0;
  __syncwarp();
  for (int base = 0; base < cap; base += 32) {
    int key = T[base + lane];
    unsigned m = __ballot_sync(0xffffffffu, key >= 0);
    int pos = nlist[wid] + __popc(m & ((1u << lane) - 1u));
    if (key >= 0) Ls[pos] = key;
    __syncwarp();
    if (lane == 0) nlist[wid] += __popc(m);
    __syncwarp();
  }
  const int nk = nlist[wid];
  const int off = crp[row];
  for (int q = lane; q < nk; q += 32) {
    int key = Ls[q];
    int rank = 0;
    for (int r = 0; r < nk; ++r) rank += Ls[r] < key;
    ccol[off + rank] = key;
  }
}

// lanes per A entry in the symbolic phase: the power of two at or above B's mean row length
static int lanes_per_entry(const DBsr& B) {
  const int64_t mean = B.nbr > 0 ? (B.nnzb + B.nbr - 1) / B.nbr : 1;
  int l = 1;
  while (l < 32 && l < mean) l <<= 1;
  return l;
}

// ---- SpGEMM over work units.  A unit is a range [ue0, ue1) of A entries of one C row urow
// (without unit tables: unit u is the whole row u).  Products with few C rows (the Galerkin
// products of the coarse levels) split their long rows over several units, so that enough warps
// work at once; the split rows are added up afterwards in unit order (deterministic).
constexpr int kSplitRows = 8192;          // products with fewer C rows use unit tables
constexpr int kTargetUnits = 4096;        // about this many units per split product
constexpr int kUnitSmem = 96 * 1024;      // shared memory per CTA for the row accumulators
constexpr size_t kUnitSmemWarp = 8 * 1024; // largest row accumulator per warp in shared memory

// symbolic phase of a split product: bm[row * wpr + c / 32] gets bit c % 32 for every column c
// of B reached from the unit's A entries (a set union, so the result does not depend on order)
__global__ void k_sym_bitmap(int nunits, const int* __restrict__ urow, const int* __restrict__ ue0,
                             const int* __restrict__ ue1, const int* __restrict__ acol, const int* __restrict__ brp,
                             const int* __restrict__ bcol, int wpr, unsigned* __restrict__ bm) {
  const int lane = threadIdx.x & 31;
  const int u = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (u >= nunits) return;
  unsigned* b = bm + (int64_t)urow[u] * wpr;
  for (int e = ue0[u]; e < ue1[u]; ++e) {
    const int k = acol[e];
    for (int t = brp[k] + lane; t < brp[k + 1]; t += 32) {
      const int c = bcol[t];
      atomicOr(b + (c >> 5), 1u << (c & 31));
    }
  }
}
// per row (one warp): the number of set bits into cnt[row], or with ccol the set columns in
// ascending order at ccol[crp[row]...]
__global__ void k_bitmap_cols(int nrow, int wpr, const unsigned* __restrict__ bm, int* __restrict__ cnt,
                              const int* __restrict__ crp, int* __restrict__ ccol) {
  const int lane = threadIdx.x & 31;
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (row >= nrow) return;
  const unsigned* b = bm + (int64_t)row * wpr;
  int total = 0;
  const int base = ccol ? crp[row] : 0;
  for (int w0 = 0; w0 < wpr; w0 += 32) {
    unsigned word = w0 + lane < wpr ? b[w0 + lane] : 0u;
    const int c = __popc(word);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (ccol) {
      int pos = base + total + incl - c;
      while (word) {
        const int bit = __ffs(word) - 1;
        ccol[pos++] = (w0 + lane) * 32 + bit;
        word &= word - 1u;
      }
    }
    total += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (!ccol && lane == 0) cnt[row] = total;
}
__global__ void k_row_maxlen(int nrow, const int* __restrict__ rp, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nrow) atomicMax(out, rp[i + 1] - rp[i]);
}
// numeric phase: one warp per unit accumulates its products into a zeroed copy of the C row and
// leaves the row in cval, or, for a split row, its partial in scratch + uout[u].  For every A
// entry (in order) the B row is taken 32 entries at a time: each lane finds the C position of
// one B entry's column, then the lanes share the (B entry, output element) work items; items
// of one group touch distinct C values (a B row has distinct columns).  SMEM: the copy lives in shared memory and is
// written out at the end; otherwise the warp accumulates in place in global memory (rows too
// long for enough warps per CTA).
// SYM (square blocks, C known to be block-symmetric): only the blocks on and above the diagonal
// are formed (B entries with a column below the row are skipped before the work items are
// dealt out); k_sym_mirror then fills the lower blocks with the transposed upper ones.
template <int BR, int BK, int BC, bool SMEM, bool SYM>
__global__ void __launch_bounds__(256)
k_spgemm_units(int nunits, const int* __restrict__ urow, const int* __restrict__ ue0, const int* __restrict__ ue1,
               const int64_t* __restrict__ uout, const int* __restrict__ arp, const int* __restrict__ acol,
               const double* __restrict__ aval, const int* __restrict__ brp, const int* __restrict__ bcol,
               const double* __restrict__ bval, const int* __restrict__ crp, const int* __restrict__ ccol,
               double* __restrict__ cval, double* __restrict__ scratch, int cmax, int cache_cols) {
  constexpr int NQ = BR * BC;
  extern __shared__ double sp_acc[];
  __shared__ int taken[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int u = blockIdx.x * nw + wid;
  if (u >= nunits) return;
  const int row = urow ? urow[u] : u;
  const int e0 = urow ? ue0[u] : arp[row], e1 = urow ? ue1[u] : arp[row + 1];
  const int c0 = crp[row], c1 = crp[row + 1];
  const int len = c1 - c0;
  double* out = (uout == nullptr || uout[u] < 0) ? cval + (int64_t)c0 * NQ : scratch + uout[u];
  double* acc = SMEM ? sp_acc + (size_t)wid * cmax * NQ : out;
  for (int q = lane; q < len * NQ; q += 32) acc[q] = 0.0;
  // the C row's columns, searched once per B entry, from shared memory when they fit
  const int* cs = ccol + c0;
  if (cache_cols) {
    int* cc = reinterpret_cast<int*>(sp_acc + (SMEM ? (size_t)nw * cmax * NQ : 0)) + (size_t)wid * cmax;
    for (int q = lane; q < len; q += 32) cc[q] = ccol[c0 + q];
    cs = cc;
  }
  __syncwarp();
  for (int e = e0; e < e1; ++e) {
    const int k = acol[e];
    const double* ae = aval + (int64_t)e * BR * BK;
    const int t0 = brp[k], t1 = brp[k + 1];
    for (int tc = t0; tc < t1; tc += 32) {
      int pos = 0;
      bool use = false;
      if (tc + lane < t1) {
        const int c = bcol[tc + lane];
        use = !SYM || c >= row;
        if (use) {
          int lo = 0, hi = len - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cs[mid] < c) lo = mid + 1;
            else hi = mid;
          }
          pos = lo;
        }
      }
      // the entries taken (all of them unless SYM), listed in lane order
      const unsigned take = __ballot_sync(0xffffffffu, use);
      const int nt = __popc(take);
      if (use) taken[wid][__popc(take & ((1u << lane) - 1u))] = lane;
      __syncwarp();
      for (int wb = 0; wb < nt * NQ; wb += 32) {
        const int w = wb + lane;
        const int t = w / NQ;
        const int src = t < nt ? taken[wid][t] : 0;   // lane holding the t-th entry taken
        const int p = __shfl_sync(0xffffffffu, pos, src);
        if (w < nt * NQ) {
          const int qe = w - t * NQ;
          const int i = qe / BC, j = qe - i * BC;
          const double* bb = bval + (int64_t)(tc + src) * BK * BC + j;
          const double* ai = ae + i * BK;
          double sacc = acc[p * NQ + qe];
#pragma unroll
          for (int m = 0; m < BK; ++m) sacc = fma(__ldg(ai + m), __ldg(bb + m * BC), sacc);
          acc[p * NQ + qe] = sacc;
        }
      }
      __syncwarp();
    }
  }
  if (SMEM)
    for (int q = lane; q < len * NQ; q += 32) out[q] = acc[q];
}
// rows split over units [su0[r], su1[r]): C row = sum of the partials in unit order; one thread
// per value of a split row (grid.y = split row)
__global__ void k_spgemm_reduce(int nsplit, const int* __restrict__ srow, const int* __restrict__ su0,
                                const int* __restrict__ su1, const int64_t* __restrict__ uout,
                                const int* __restrict__ crp, int nq, const double* __restrict__ scratch,
                                double* __restrict__ cval) {
  const int r = blockIdx.y;
  if (r >= nsplit) return;
  const int row = srow[r];
  const int64_t c0 = crp[row];
  const int len = (crp[row + 1] - crp[row]) * nq;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= len) return;
  double t = 0.0;
  for (int u = su0[r]; u < su1[r]; ++u) t += scratch[uout[u] + q];
  cval[c0 * nq + q] = t;
}

// lower blocks of a block-symmetric product: C[I][J] = C[J][I]^T for J < I (one warp per row)
template <int B>
__global__ void k_sym_mirror(int nrow, const int* __restrict__ crp, const int* __restrict__ ccol,
                             double* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const int I = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (I >= nrow) return;
  for (int e = crp[I] + lane; e < crp[I + 1]; e += 32) {
    const int J = ccol[e];
    if (J >= I) continue;
    int lo = crp[J], hi = crp[J + 1] - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ccol[mid] < I) lo = mid + 1;
      else hi = mid;
    }
    const double* up = cval + (int64_t)lo * B * B;
    double* dn = cval + (int64_t)e * B * B;
    for (int r = 0; r < B; ++r)
      for (int c = 0; c < B; ++c) dn[r * B + c] = up[c * B + r];
  }
}

// Work units of a split product (host tables, copied to the device).
struct SpUnits {
  std::vector<int> row, e0, e1, srow, su0, su1;
  std::vector<int64_t> out;
  int64_t scratch = 0;
  DBuf<int> d_row, d_e0, d_e1, d_srow, d_su0, d_su1;
  DBuf<int64_t> d_out;
};
// rows longer than seg A entries are cut into pieces of at most seg entries
static void build_units(const std::vector<int>& arp, int seg, SpUnits& U) {
  const int n = (int)arp.size() - 1;
  for (int r = 0; r < n; ++r) {
    const int a = arp[r], b = arp[r + 1];
    if (b - a <= seg) {
      U.row.push_back(r);
      U.e0.push_back(a);
      U.e1.push_back(b);
      continue;
    }
    U.srow.push_back(r);
    U.su0.push_back((int)U.row.size());
    for (int e = a; e < b; e += seg) {
      U.row.push_back(r);
      U.e0.push_back(e);
      U.e1.push_back(std::min(b, e + seg));
    }
    U.su1.push_back((int)U.row.size());
  }
}
template <class T>
static int upload(DBuf<T>& d, const std::vector<T>& h, cudaStream_t s) {
  AMGC_TRY(d.alloc(std::max<size_t>(h.size(), 1)));
  if (!h.empty()) AMGC_CUDA_TRY(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return AMGC_OK;
}

// C values: with shared-memory row accumulators when the longest C row fits (cmax), over the
// unit tables U when the product is split, else with the global-memory accumulation kernel.
template <int BR, int BK, int BC, bool SYM = false>
static int spgemm_numeric(const DBsr& A, const DBsr& B, DBsr& C, int cmax, SpUnits* U, cudaStream_t s) {
  constexpr int NQ = BR * BC;
  const size_t per_warp = (size_t)std::max(cmax, 1) * NQ * sizeof(double);
  // shared-memory accumulators only for short C rows (eight warps in at most 64 KB, so that
  // three CTAs share an SM); longer rows accumulate in global memory, where more warps per SM
  // hide the latency of the position searches better than shared memory saves
  const bool smem_acc = per_warp <= kUnitSmemWarp;
  const int wpb = smem_acc ? 8 : kGemmWarps;
  // plus each warp's copy of its C row's columns when that stays within the CTA's budget
  const size_t acc_bytes = smem_acc ? (size_t)wpb * per_warp : 0;
  const size_t col_bytes = (size_t)wpb * std::max(cmax, 1) * sizeof(int);
  const int cache_cols = acc_bytes + col_bytes <= (size_t)kUnitSmem ? 1 : 0;
  const size_t smem = acc_bytes + (cache_cols ? col_bytes : 0);
  auto kern = smem_acc ? k_spgemm_units<BR, BK, BC, true, SYM> : k_spgemm_units<BR, BK, BC, false, SYM>;
  // (the dynamic limit is raised for every launch: the kernel's static shared memory counts
  // against the default 48 KB too)
  AMGC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kUnitSmem));
  DBuf<double> scratch;
  if (U) {
    const int nu = (int)U->row.size();
    if (U->scratch > 0) AMGC_TRY(scratch.alloc((size_t)U->scratch));
    AMGC_LAUNCH(kern<<<div_up(nu, wpb), wpb * 32, smem, s>>>(
        nu, U->d_row.p, U->d_e0.p, U->d_e1.p, U->d_out.p, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p,
        C.rowptr.p, C.col.p, C.val.p, scratch.p, cmax, cache_cols));
    const int ns = (int)U->srow.size();
    if (ns > 0 && cmax > 0)   // (an empty product, cmax = 0, has nothing to add up)
      AMGC_LAUNCH(k_spgemm_reduce<<<dim3(div_up((int64_t)cmax * NQ, 128), ns), 128, 0, s>>>(
          ns, U->d_srow.p, U->d_su0.p, U->d_su1.p, U->d_out.p, C.rowptr.p, NQ, scratch.p, C.val.p));
  } else {
    AMGC_LAUNCH(kern<<<div_up(A.nbr, wpb), wpb * 32, smem, s>>>(
        A.nbr, nullptr, nullptr, nullptr, nullptr, A.rowptr.p, A.col.p, A.val.p, B.rowptr.p, B.col.p, B.val.p,
        C.rowptr.p, C.col.p, C.val.p, nullptr, cmax, cache_cols));
  }
  if (SYM)
    AMGC_LAUNCH(k_sym_mirror<BR><<<div_up((int64_t)A.nbr * 32, 128), 128, 0, s>>>(A.nbr, C.rowptr.p, C.col.p, C.val.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// sym: C = A B is known to be block-symmetric (a Galerkin product P^T K P): square blocks only
int spgemm(amgc_hierarchy* h, const DBsr& A, const DBsr& B, DBsr& C, bool sym) {
  cudaStream_t s = h->stream;
  if (A.bc != B.br || A.nbc != B.nbr) {
    set_error("spgemm: shape mismatch");
    return AMGC_EINVAL;
  }
  C.nbr = A.nbr;
  C.nbc = B.nbc;
  C.br = A.br;
  C.bc = B.bc;
  AMGC_TRY(C.rowptr.alloc(A.nbr + 1));
  AMGC_CUDA_TRY(cudaMemsetAsync(C.rowptr.p, 0, (A.nbr + 1) * sizeof(int), s));
  const int wpr = (B.nbc + 31) / 32;
  // few C rows: unit tables (long rows split) and a bitmap symbolic phase
  const bool split = A.nbr > 0 && A.nbr < kSplitRows && (int64_t)A.nbr * wpr <= (int64_t)(64 << 20);
  std::unique_ptr<SpUnits> U;
  DBuf<unsigned> bm;
  const int g = div_up(A.nbr, kGemmWarps);
  if (split) {
    U.reset(new SpUnits());
    std::vector<int> arp(A.nbr + 1);
    AMGC_CUDA_TRY(cudaMemcpyAsync(arp.data(), A.rowptr.p, (A.nbr + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nnza = arp[A.nbr];
    const int seg = (int)std::max<int64_t>(4, (nnza + kTargetUnits - 1) / kTargetUnits);
    build_units(arp, seg, *U);
    AMGC_TRY(upload(U->d_row, U->row, s));
    AMGC_TRY(upload(U->d_e0, U->e0, s));
    AMGC_TRY(upload(U->d_e1, U->e1, s));
    AMGC_TRY(bm.alloc((size_t)A.nbr * std::max(wpr, 1)));
    AMGC_CUDA_TRY(cudaMemsetAsync(bm.p, 0, (size_t)A.nbr * std::max(wpr, 1) * sizeof(unsigned), s));
    const int nu = (int)U->row.size();
    AMGC_LAUNCH(k_sym_bitmap<<<div_up((int64_t)nu * 32, 256), 256, 0, s>>>(nu, U->d_row.p, U->d_e0.p, U->d_e1.p,
                                                                            A.col.p, B.rowptr.p, B.col.p, wpr, bm.p));
    AMGC_LAUNCH(k_bitmap_cols<<<div_up((int64_t)A.nbr * 32, 256), 256, 0, s>>>(A.nbr, wpr, bm.p, C.rowptr.p, nullptr,
                                                                                 nullptr));
  } else if (A.nbr > 0) {
    AMGC_LAUNCH(k_spgemm_symbolic<0><<<g, kGemmWarps * 32, 0, s>>>(A.nbr, lanes_per_entry(B), A.rowptr.p, A.col.p,
                                                                  B.rowptr.p, B.col.p,
                                                                  C.rowptr.p, nullptr, nullptr, h->status.p));
  }
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(check_status(h, "spgemm symbolic"));
  int nnz = 0;
  AMGC_TRY(exclusive_scan(C.rowptr.p, C.rowptr.p, A.nbr + 1, s, &nnz));
  C.nnzb = nnz;
  AMGC_TRY(C.col.alloc(std::max(nnz, 1)));
  AMGC_TRY(C.val.alloc((size_t)std::max(nnz, 1) * C.br * C.bc));
  if (A.nbr == 0) return AMGC_OK;
  int cmax = 0;
  if (split) {
    AMGC_LAUNCH(k_bitmap_cols<<<div_up((int64_t)A.nbr * 32, 256), 256, 0, s>>>(A.nbr, wpr, bm.p, nullptr, C.rowptr.p,
                                                                                 C.col.p));
    // C row lengths give the scratch slices of the split rows
    std::vector<int> crp(A.nbr + 1);
    AMGC_CUDA_TRY(cudaMemcpyAsync(crp.data(), C.rowptr.p, (A.nbr + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
    for (int r = 0; r < A.nbr; ++r) cmax = std::max(cmax, crp[r + 1] - crp[r]);
    const int64_t nq = (int64_t)C.br * C.bc;
    U->out.assign(U->row.size(), -1);
    for (size_t q = 0; q < U->srow.size(); ++q) {
      const int r = U->srow[q];
      for (int u = U->su0[q]; u < U->su1[q]; ++u) {
        U->out[u] = U->scratch;
        U->scratch += (int64_t)(crp[r + 1] - crp[r]) * nq;
      }
    }
    AMGC_TRY(upload(U->d_out, U->out, s));
    AMGC_TRY(upload(U->d_srow, U->srow, s));
    AMGC_TRY(upload(U->d_su0, U->su0, s));
    AMGC_TRY(upload(U->d_su1, U->su1, s));
  } else {
    AMGC_LAUNCH(k_spgemm_symbolic<1><<<g, kGemmWarps * 32, 0, s>>>(A.nbr, lanes_per_entry(B), A.rowptr.p, A.col.p,
                                                                  B.rowptr.p, B.col.p,
                                                                  nullptr, C.rowptr.p, C.col.p, h->status.p));
    DBuf<int> mx;
    AMGC_TRY(mx.alloc(1));
    AMGC_CUDA_TRY(cudaMemsetAsync(mx.p, 0, sizeof(int), s));
    AMGC_LAUNCH(k_row_maxlen<<<div_up(A.nbr, 256), 256, 0, s>>>(A.nbr, C.rowptr.p, mx.p));
    AMGC_CUDA_TRY(cudaMemcpyAsync(&cmax, mx.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  }
  AMGC_CUDA_TRY(cudaGetLastError());
  const int br = A.br, bk = A.bc, bc = B.bc;
  SpUnits* up = U.get();
  if (sym && br == 6 && bk == 3 && bc == 6) return spgemm_numeric<6, 3, 6, true>(A, B, C, cmax, up, s);
  if (sym && br == 6 && bk == 6 && bc == 6) return spgemm_numeric<6, 6, 6, true>(A, B, C, cmax, up, s);
#define AMGC_GEMM_CASE(R, K, C_)                                   \
  if (br == R && bk == K && bc == C_) return spgemm_numeric<R, K, C_>(A, B, C, cmax, up, s);
  AMGC_GEMM_CASE(3, 3, 6)
  AMGC_GEMM_CASE(6, 3, 6)
  AMGC_GEMM_CASE(3, 3, 3)
  AMGC_GEMM_CASE(6, 3, 3)
  AMGC_GEMM_CASE(6, 6, 6)
  AMGC_GEMM_CASE(6, 6, 3)
  AMGC_GEMM_CASE(3, 6, 6)
  AMGC_GEMM_CASE(3, 6, 3)
#undef AMGC_GEMM_CASE
  set_error("spgemm: unsupported block shape");
  return AMGC_EINVAL;
}

// ======================================================================== BSR transpose
__global__ void k_tr_count(int64_t nnzb, const int* __restrict__ col, int* __restrict__ cnt) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nnzb) atomicAdd(cnt + col[e], 1);
}
__global__ void k_tr_scatter(int nbr, const int* __restrict__ rp, const int* __restrict__ col, int* __restrict__ cur,
                             int* __restrict__ trow, int* __restrict__ src) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int p = atomicAdd(cur + col[e], 1);
    trow[p] = i;
    src[p] = e;
  }
}
__global__ void k_tr_values(int64_t nnzb, int br, int bc, const int* __restrict__ src, const double* __restrict__ val,
                            double* __restrict__ tval) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  const double* a = val + (int64_t)src[e] * br * bc;
  double* t = tval + e * br * bc;
  for (int i = 0; i < br; ++i)
    for (int j = 0; j < bc; ++j) t[j * br + i] = a[i * bc + j];
}

static int bsr_transpose(amgc_hierarchy* h, const DBsr& A, DBsr& T) {
  cudaStream_t s = h->stream;
  T.nbr = A.nbc;
  T.nbc = A.nbr;
  T.br = A.bc;
  T.bc = A.br;
  T.nnzb = A.nnzb;
  AMGC_TRY(T.rowptr.alloc(A.nbc + 1));
  AMGC_TRY(T.col.alloc(std::max<int64_t>(A.nnzb, 1)));
  AMGC_TRY(T.val.alloc((size_t)std::max<int64_t>(A.nnzb, 1) * A.br * A.bc));
  DBuf<int> cur, src;
  AMGC_TRY(cur.alloc(A.nbc + 1));
  AMGC_TRY(src.alloc(std::max<int64_t>(A.nnzb, 1)));
  AMGC_CUDA_TRY(cudaMemsetAsync(T.rowptr.p, 0, (A.nbc + 1) * sizeof(int), s));
  if (A.nnzb > 0) AMGC_LAUNCH(k_tr_count<<<div_up(A.nnzb, 256), 256, 0, s>>>(A.nnzb, A.col.p, T.rowptr.p));
  AMGC_TRY(exclusive_scan(T.rowptr.p, T.rowptr.p, A.nbc + 1, s, nullptr));
  AMGC_LAUNCH(k_copy_int<<<div_up(A.nbc + 1, 256), 256, 0, s>>>(A.nbc + 1, T.rowptr.p, cur.p));
  if (A.nbr > 0) AMGC_LAUNCH(k_tr_scatter<<<div_up(A.nbr, 256), 256, 0, s>>>(A.nbr, A.rowptr.p, A.col.p, cur.p, T.col.p, src.p));
  if (A.nbc > 0) AMGC_LAUNCH(k_sort_segments_warp<<<div_up(A.nbc, kSortWarps), kSortWarps * 32, 0, s>>>(A.nbc, T.rowptr.p, T.col.p, src.p));
  if (A.nnzb > 0) AMGC_LAUNCH(k_tr_values<<<div_up(A.nnzb, 256), 256, 0, s>>>(A.nnzb, A.br, A.bc, src.p, A.val.p, T.val.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

// ======================================================================== smoothed prolongator
// P = P-hat - omega D^{-1} (K P-hat) on the pattern of K P-hat (K holds its diagonal blocks,
// so that pattern contains P-hat's).  One warp per node row; the lanes take the row's values
// (its blocks are contiguous), so that loads and stores are coalesced.
template <int BU>
__global__ void k_sa_values(int nn, const int* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ agg,
                            const double* __restrict__ phat, const double* __restrict__ dinv, double omega,
                            const double* __restrict__ omega_dof, double* __restrict__ val) {
  constexpr int NQ = BU * 6;
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= nn) return;
  const int e0 = rp[i], nq = (rp[i + 1] - e0) * NQ;
  const int a = agg[i];
  double* v = val + (int64_t)e0 * NQ;
  for (int q = lane; q < nq; q += 32) {
    const int eb = q / NQ;
    const int w = q - eb * NQ;
    const int r = w / 6, c = w - r * 6;
    const int64_t dof = (int64_t)i * BU + r;
    const double d = (omega_dof ? omega_dof[dof] : omega) * dinv[dof];
    const double p = col[e0 + eb] == a ? phat[dof * 6 + c] : 0.0;
    v[q] = p - d * v[q];
  }
}

// ======================================================================== smoother data
// Pointwise diagonal of K, its inverse and the inverse of A~ (the diagonal, or with SIMPLEC the
// absolute row sums).  One thread per node row: the diagonal block is found by binary search
// (columns ascending), and only SIMPLEC walks the whole row.
template <int BU>
__global__ void k_diag(int nn, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                       int simplec, double* __restrict__ kdiag, double* __restrict__ dinv, double* __restrict__ atinv,
                       int* st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int e0 = rp[i], e1 = rp[i + 1];
  int lo = e0, hi = e1 - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (col[mid] < i) lo = mid + 1;
    else hi = mid;
  }
  const bool found = e1 > e0 && col[lo] == i;
  if (!found) set_status(st, ST_NO_DIAG);
  double as[BU];
#pragma unroll
  for (int r = 0; r < BU; ++r) as[r] = 0.0;
  if (simplec)
    for (int e = e0; e < e1; ++e) {
      const double* v = val + (int64_t)e * BU * BU;
#pragma unroll
      for (int r = 0; r < BU; ++r)
#pragma unroll
        for (int c = 0; c < BU; ++c) as[r] += fabs(v[r * BU + c]);
    }
#pragma unroll
  for (int r = 0; r < BU; ++r) {
    const double dg = found ? val[((int64_t)lo * BU + r) * BU + r] : 0.0;
    if (!(dg > 0.0) || !isfinite(dg)) set_status(st, ST_SINGULAR);
    kdiag[(int64_t)i * BU + r] = dg;
    dinv[(int64_t)i * BU + r] = 1.0 / dg;
    atinv[(int64_t)i * BU + r] = 1.0 / (simplec ? as[r] : dg);
  }
}
// S_l = Z_l + sum_i B2[l,i] diag(atinv_i) B1[i,l]; Sinv_l = S_l^{-1}.  One warp per multiplier
// node: the lanes take the B2 entries of the row (coarse rows have many), the nine partial sums
// are added across the warp, and lane 0 inverts the block.
template <int BU>
__global__ void k_schur(int nl, const int* __restrict__ rp2, const int* __restrict__ c2, const double* __restrict__ v2,
                        const int* __restrict__ rp1, const int* __restrict__ c1, const double* __restrict__ v1,
                        const double* __restrict__ atinv, const double* __restrict__ Z, double* __restrict__ Sinv, int* st) {
  const int lane = threadIdx.x & 31;
  const int l = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (l >= nl) return;
  double S[9];
  for (int t = 0; t < 9; ++t) S[t] = 0.0;
  for (int e = rp2[l] + lane; e < rp2[l + 1]; e += 32) {
    const int i = c2[e];
    // find block (i, l) of B1
    int lo = rp1[i], hi = rp1[i + 1] - 1, pos = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1;
      int c = c1[mid];
      if (c == l) { pos = mid; break; }
      if (c < l) lo = mid + 1;
      else hi = mid - 1;
    }
    if (pos < 0) continue;
    const double* b2 = v2 + (int64_t)e * 3 * BU;     // 3 x BU
    const double* b1 = v1 + (int64_t)pos * BU * 3;   // BU x 3
    for (int m = 0; m < BU; ++m) {
      const double a = atinv[(int64_t)i * BU + m];
      for (int r = 0; r < 3; ++r) {
        const double x = b2[r * BU + m] * a;
        for (int c = 0; c < 3; ++c) S[r * 3 + c] = fma(x, b1[m * 3 + c], S[r * 3 + c]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 9; ++t) S[t] = warp_sum(S[t]);
  if (lane != 0) return;
  for (int t = 0; t < 9; ++t) S[t] += Z[(int64_t)l * 9 + t];
  // 3x3 inverse by cofactors
  const double c00 = S[4] * S[8] - S[5] * S[7];
  const double c01 = S[5] * S[6] - S[3] * S[8];
  const double c02 = S[3] * S[7] - S[4] * S[6];
  const double det = S[0] * c00 + S[1] * c01 + S[2] * c02;
  double nrm = 0.0;
  for (int t = 0; t < 9; ++t) nrm = fmax(nrm, fabs(S[t]));
  if (!(fabs(det) > 1e-14 * nrm * nrm * nrm) || !isfinite(det)) {
    set_status(st, ST_SINGULAR);
    return;
  }
  const double id = 1.0 / det;
  double* o = Sinv + (int64_t)l * 9;
  o[0] = c00 * id;
  o[1] = (S[2] * S[7] - S[1] * S[8]) * id;
  o[2] = (S[1] * S[5] - S[2] * S[4]) * id;
  o[3] = c01 * id;
  o[4] = (S[0] * S[8] - S[2] * S[6]) * id;
  o[5] = (S[2] * S[3] - S[0] * S[5]) * id;
  o[6] = c02 * id;
  o[7] = (S[1] * S[6] - S[0] * S[7]) * id;
  o[8] = (S[0] * S[4] - S[1] * S[3]) * id;
}
__global__ void k_nonempty(int n, const int* __restrict__ rp, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = rp[i + 1] > rp[i] ? 1 : 0;
}
__global__ void k_compact(int n, const int* __restrict__ flag_rp, const int* __restrict__ rank, int* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag_rp[i + 1] > flag_rp[i]) out[rank[i]] = i;
}

__global__ void k_scale_omega(int n, const double* __restrict__ dinv, double omega, const double* __restrict__ wdof,
                              double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (wdof ? wdof[i] : omega) * dinv[i];
}
__global__ void k_key_base(int ni, const int* __restrict__ nptr, int* __restrict__ base) {
  const int q = blockIdx.x;
  if (q >= ni) return;
  for (int i = nptr[q] + threadIdx.x; i < nptr[q + 1]; i += blockDim.x) base[i] = nptr[q];
}
// batched levels: first node of each node's instance (MIS-2 keys)
static int build_key_base(amgc_hierarchy* h, Level& L) {
  if (h->n_inst <= 1) return AMGC_OK;
  cudaStream_t s = h->stream;
  DBuf<int> dptr;
  AMGC_TRY(dptr.alloc(h->n_inst + 1));
  AMGC_CUDA_TRY(cudaMemcpyAsync(dptr.p, L.nptr.data(), (h->n_inst + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_TRY(L.key_base.alloc(std::max(L.nn, 1)));
  AMGC_LAUNCH(k_key_base<<<h->n_inst, 256, 0, s>>>(h->n_inst, dptr.p, L.key_base.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

static int alloc_work(Level& L) {
  const int n = L.rows();
  AMGC_TRY(L.x.alloc(std::max(n, 1)));
  AMGC_TRY(L.b.alloc(std::max(n, 1)));
  AMGC_TRY(L.r.alloc(std::max(n, 1)));
  AMGC_TRY(L.t.alloc(std::max(n, 1)));
  AMGC_TRY(L.dlam.alloc(std::max(3 * L.nl, 1)));
  return AMGC_OK;
}

static int smoother_rest(amgc_hierarchy* h, Level& L);

int smoother_setup(amgc_hierarchy* h, int l) {
  cudaStream_t s = h->stream;
  Level& L = h->L[l];
  const int nu = L.nu();
  AMGC_TRY(L.kdiag.alloc(nu));
  AMGC_TRY(L.dinv.alloc(nu));
  AMGC_TRY(L.atinv.alloc(nu));
  if (L.bu == 3)
    AMGC_LAUNCH(k_diag<3><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p, h->opts.simplec, L.kdiag.p,
                                                L.dinv.p, L.atinv.p, h->status.p));
  else
    AMGC_LAUNCH(k_diag<6><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p, h->opts.simplec, L.kdiag.p,
                                                L.dinv.p, L.atinv.p, h->status.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(check_status(h, "K diagonal"));
  AMGC_TRY(L.Sinv.alloc((size_t)std::max(L.nl, 1) * 9));
  if (L.nl > 0) {
    if (L.bu == 3)
      AMGC_LAUNCH(k_schur<3><<<div_up((int64_t)L.nl * 32, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, L.B1.rowptr.p,
                                                   L.B1.col.p, L.B1.val.p, L.atinv.p, L.Z.p, L.Sinv.p, h->status.p));
    else
      AMGC_LAUNCH(k_schur<6><<<div_up((int64_t)L.nl * 32, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, L.B1.rowptr.p,
                                                   L.B1.col.p, L.B1.val.p, L.atinv.p, L.Z.p, L.Sinv.p, h->status.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    AMGC_TRY(check_status(h, "Schur blocks"));
  }
  // rows of B1 with entries
  DBuf<int> flag;
  AMGC_TRY(flag.alloc(L.nn + 1));
  AMGC_LAUNCH(k_nonempty<<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B1.rowptr.p, flag.p));
  int cnt = 0;
  AMGC_TRY(exclusive_scan(flag.p, flag.p, L.nn, s, &cnt));
  L.n_b1_rows = cnt;
  AMGC_TRY(L.b1_rows.alloc(std::max(cnt, 1)));
  AMGC_LAUNCH(k_compact<<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B1.rowptr.p, flag.p, L.b1_rows.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  if (L.lam_max == 0.0) {
    if (h->n_inst > 1) {
      AMGC_TRY(lambda_max_instances(h, L, L.inst_lam_max));
      L.lam_max = L.inst_lam_max[0];
    } else {
      // single instance: the power iteration runs on the auxiliary stream; the rest of the
      // smoother data waits for it in smoother_finish
      AMGC_TRY(lambda_max_start(h, L));
      L.smoother_pending = true;
      return AMGC_OK;
    }
  }
  return smoother_rest(h, L);
}

// Joins a pending lambda_max of level l and completes its smoother data (no-op otherwise).
int smoother_finish(amgc_hierarchy* h, int l) {
  Level& L = h->L[l];
  if (!L.smoother_pending) return AMGC_OK;
  L.smoother_pending = false;
  AMGC_TRY(lambda_max_finish(h, L, &L.lam_max));
  return smoother_rest(h, L);
}

// omega_J, the scaled Jacobi diagonal, the Schur-step damping and the work vectors of a level
// whose lambda_max is known
static int smoother_rest(amgc_hierarchy* h, Level& L) {
  cudaStream_t s = h->stream;
  const int nu = L.nu();
  L.omega_j = h->opts.jacobi_omega > 0.0 ? h->opts.jacobi_omega : (4.0 / 3.0) / L.lam_max;
  // omega_J D^-1 per DOF (omega_J per instance when batched)
  {
    std::vector<double> w;
    const double* wp = nullptr;
    if (h->n_inst > 1) {
      w.resize(L.nu());
      for (int q = 0; q < h->n_inst; ++q) {
        const double om = h->opts.jacobi_omega > 0.0 ? h->opts.jacobi_omega : (4.0 / 3.0) / L.inst_lam_max[q];
        for (int i = L.bu * L.nptr[q]; i < L.bu * L.nptr[q + 1]; ++i) w[i] = om;
      }
      wp = w.data();
    }
    AMGC_TRY(L.jdinv.alloc(nu));
    DBuf<double> wd;
    if (wp) {
      AMGC_TRY(wd.alloc(nu));
      AMGC_CUDA_TRY(cudaMemcpyAsync(wd.p, wp, nu * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    AMGC_LAUNCH(k_scale_omega<<<div_up(nu, 256), 256, 0, s>>>(nu, L.dinv.p, L.omega_j, wd.p, L.jdinv.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (h->opts.schur_damping && L.nl > 0) AMGC_TRY(schur_damping_setup(h, L));
  AMGC_TRY(alloc_work(L));
  return AMGC_OK;
}

// ======================================================================== SELL-32 copies
// Slice sl holds the block rows at SELL positions 32 sl .. 32 sl + 31, padded to the longest of
// them.  Where row lengths vary (the prolongators, the coarse K), the rows are first sorted by
// length within windows of kSellWindow rows (perm: position -> row, longest first, ties by row),
// so that a slice holds rows of nearly equal length and little padding; the applies write each
// row at its own index, and a row's sum runs over its blocks in the same order either way.
constexpr int kSellWindow = 1024;
__global__ void __launch_bounds__(kSellWindow)
k_sell_sort(int nbr, const int* __restrict__ rp, int* __restrict__ perm) {
  __shared__ unsigned key[kSellWindow];
  const int w0 = blockIdx.x * kSellWindow;
  const int t = threadIdx.x;
  const int row = w0 + t;
  // key: (2^20 - 1 - length) above the local index, so ascending keys put long rows first and
  // equal lengths in row order; positions past the last row sort to the end
  if (row < nbr) {
    const int len = min(rp[row + 1] - rp[row], (1 << 20) - 1);
    key[t] = ((unsigned)((1 << 20) - 1 - len) << 11) | (unsigned)t;
  } else {
    key[t] = 0xffffffffu;
  }
  __syncthreads();
  // bitonic sort of the window's keys, ascending
  for (int k = 2; k <= kSellWindow; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int q = t ^ j;
      if (q > t) {
        const unsigned a = key[t], b = key[q];
        const bool up = (t & k) == 0;
        if ((a > b) == up) {
          key[t] = b;
          key[q] = a;
        }
      }
      __syncthreads();
    }
  }
  if (row < nbr) perm[row] = w0 + (int)(key[t] & 2047u);
}
__global__ void k_sell_len(int nbr, int nslice, const int* __restrict__ rp, const int* __restrict__ perm,
                           int* __restrict__ len) {
  int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslice) return;
  int m = 0;
  for (int p = sl * 32; p < sl * 32 + 32 && p < nbr; ++p) {
    const int r = perm ? perm[p] : p;
    m = max(m, rp[r + 1] - rp[r]);
  }
  len[sl] = m;
}
__global__ void k_sell_fill(int nbr, int nslice, int bs, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ val, const int* __restrict__ off, const int* __restrict__ len,
                            const int* __restrict__ perm, int* __restrict__ scol, double* __restrict__ sval) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= nslice * 32) return;
  const int lane = pos & 31, sl = pos >> 5;
  const int64_t o = off[sl];
  const int L = len[sl];
  const int row = pos < nbr ? (perm ? perm[pos] : pos) : -1;
  const int b0 = row >= 0 ? rp[row] : 0;
  const int nb = row >= 0 ? rp[row + 1] - b0 : 0;
  for (int t = 0; t < L; ++t) {
    const int64_t ci = (o + t) * 32 + lane;
    const int64_t vi = (o + t) * bs * 32 + lane;
    if (t < nb) {
      scol[ci] = col[b0 + t];
      const double* v = val + (int64_t)(b0 + t) * bs;
      for (int k = 0; k < bs; ++k) sval[vi + 32 * k] = v[k];
    } else {
      scol[ci] = 0;
      for (int k = 0; k < bs; ++k) sval[vi + 32 * k] = 0.0;
    }
  }
}

// The fine level's 3x3 K (rows of nearly equal length, and the staged FP32 kernel reads its slices
// as rows) keeps the identity order; every other matrix is sorted by length within windows.
int build_sell_of(amgc_hierarchy* h, const DBsr& A, Sell& S) {
  cudaStream_t s = h->stream;
  const int ns = div_up(A.nbr, 32);
  const int bs = A.br * A.bc;
  S.br = A.br;
  S.bc = A.bc;
  const bool sorted = !(A.br == 3 && A.bc == 3) && A.nbr > 32;
  S.perm.release();
  if (sorted) {
    AMGC_TRY(S.perm.alloc(A.nbr));
    AMGC_LAUNCH(k_sell_sort<<<div_up(A.nbr, kSellWindow), kSellWindow, 0, s>>>(A.nbr, A.rowptr.p, S.perm.p));
  }
  AMGC_TRY(S.len.alloc(ns));
  AMGC_TRY(S.off.alloc(ns + 1));
  AMGC_LAUNCH(k_sell_len<<<div_up(ns, 128), 128, 0, s>>>(A.nbr, ns, A.rowptr.p, S.perm.p, S.len.p));
  AMGC_CUDA_TRY(cudaMemsetAsync(S.off.p, 0, (ns + 1) * sizeof(int), s));
  AMGC_LAUNCH(k_copy_int<<<div_up(ns, 256), 256, 0, s>>>(ns, S.len.p, S.off.p));
  int slots = 0;
  AMGC_TRY(exclusive_scan(S.off.p, S.off.p, ns + 1, s, &slots));
  S.slots = slots;
  AMGC_TRY(S.col.alloc((size_t)std::max(slots, 1) * 32));
  AMGC_TRY(S.val.alloc((size_t)std::max(slots, 1) * bs * 32));
  AMGC_LAUNCH(k_sell_fill<<<div_up((int64_t)ns * 32, 256), 256, 0, s>>>(A.nbr, ns, bs, A.rowptr.p, A.col.p, A.val.p,
                                                                      S.off.p, S.len.p, S.perm.p, S.col.p, S.val.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  S.nslice = ns;
  return AMGC_OK;
}

// SELL copies of the finest level's K (3x3) and, once it exists, P (3x6) for the
// thread-per-row applies; each copy is built once.
int build_sell(amgc_hierarchy* h, int l) {
  Level& L = h->L[l];
  if (L.bu != 3) return AMGC_OK;
  if (L.Ks.nslice == 0) AMGC_TRY(build_sell_of(h, L.K, L.Ks));
  if (L.P.nbr > 0 && L.Ps.nslice == 0) AMGC_TRY(build_sell_of(h, L.P, L.Ps));
  return AMGC_OK;
}

// ======================================================================== coarsening
// coarse instance boundaries: aggregates are numbered by ascending root, so instance i owns the
// aggregates whose root lies below its first node; multiplier aggregates follow the rank of
// their first coupled displacement node
__global__ void k_inst_bounds(int n_inst1, const int* __restrict__ nptr, const int* __restrict__ roots, int n_agg,
                              const int* __restrict__ mark_rank, int nn, int n_lagg, int* __restrict__ nptr_c,
                              int* __restrict__ lptr_c) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_inst1) return;
  const int b = nptr[i];
  int lo = 0, hi = n_agg;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (roots[mid] < b) lo = mid + 1;
    else hi = mid;
  }
  nptr_c[i] = lo;
  lptr_c[i] = b < nn ? mark_rank[b] : n_lagg;
}

__global__ void k_gather_body(int n, const int* __restrict__ roots, const int* __restrict__ body, int* __restrict__ out) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) out[a] = body[roots[a]];
}

int coarsen_level(amgc_hierarchy* h, int l) {
  cudaStream_t s = h->stream;
  Level& L = h->L[l];
  // --- displacement aggregates
  DBuf<int> roots;
  int n_agg = 0;
  AMGC_TRY(build_key_base(h, L));
  {
    PhaseTimer pt(h, 1);
    AMGC_TRY(mis2_aggregate(h, L, roots, &n_agg));
  }
  L.n_agg = n_agg;
  // --- multiplier aggregates (Algorithm 1)
  std::unique_ptr<PhaseTimer> ptm(new PhaseTimer(h, 2));
  DBuf<int> first, mark, lm_dnode_c;
  AMGC_TRY(first.alloc(n_agg));
  AMGC_TRY(mark.alloc(L.nn + 1));
  AMGC_TRY(L.lagg.alloc(std::max(L.nl, 1)));
  AMGC_TRY(lm_dnode_c.alloc(std::max(L.nl, 1)));
  AMGC_LAUNCH(k_fill_int<<<div_up(n_agg, 256), 256, 0, s>>>(n_agg, 0x7fffffff, first.p));
  if (L.nl > 0) AMGC_LAUNCH(k_lm_first<<<div_up(L.nl, 256), 256, 0, s>>>(L.nl, L.lm_dnode.p, L.agg.p, first.p));
  AMGC_LAUNCH(k_lm_mark<<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.agg.p, first.p, mark.p));
  int n_lagg = 0;
  AMGC_TRY(exclusive_scan(mark.p, mark.p, L.nn, s, &n_lagg));
  if (L.nl > 0)
    AMGC_LAUNCH(k_lm_assign<<<div_up(L.nl, 256), 256, 0, s>>>(L.nl, L.lm_dnode.p, L.agg.p, first.p, mark.p, L.lagg.p, lm_dnode_c.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  L.n_lagg = n_lagg;
  std::vector<int> nptr_c, lptr_c;
  if (h->n_inst > 1) {
    const int ni1 = h->n_inst + 1;
    DBuf<int> d_nptr, d_np, d_lp;
    AMGC_TRY(d_nptr.alloc(ni1));
    AMGC_TRY(d_np.alloc(ni1));
    AMGC_TRY(d_lp.alloc(ni1));
    AMGC_CUDA_TRY(cudaMemcpyAsync(d_nptr.p, L.nptr.data(), ni1 * sizeof(int), cudaMemcpyHostToDevice, s));
    AMGC_LAUNCH(k_inst_bounds<<<div_up(ni1, 128), 128, 0, s>>>(ni1, d_nptr.p, roots.p, n_agg, mark.p, L.nn, n_lagg,
                                                               d_np.p, d_lp.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    nptr_c.resize(ni1);
    lptr_c.resize(ni1);
    AMGC_CUDA_TRY(cudaMemcpyAsync(nptr_c.data(), d_np.p, ni1 * sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaMemcpyAsync(lptr_c.data(), d_lp.p, ni1 * sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  }
  ptm.reset();
  // --- tentative displacement prolongator by QR
  ptm.reset(new PhaseTimer(h, 3));
  DBuf<int> mptr, midx;
  AMGC_TRY(bucket_lists(L.nn, L.agg.p, n_agg, mptr, midx, s));
  DBsr Phat;
  Phat.nbr = L.nn; Phat.nbc = n_agg; Phat.br = L.bu; Phat.bc = 6; Phat.nnzb = L.nn;
  AMGC_TRY(Phat.rowptr.alloc(L.nn + 1));
  AMGC_TRY(Phat.col.alloc(L.nn));
  AMGC_TRY(Phat.val.alloc((size_t)L.nn * L.bu * 6));
  Level C;
  C.nn = n_agg;
  C.bu = 6;
  C.nl = n_lagg;
  C.nptr = nptr_c;
  C.lptr = lptr_c;
  AMGC_TRY(C.B.alloc((size_t)n_agg * 36));
  AMGC_LAUNCH(k_tentative_pattern<<<div_up(L.nn + 1, 256), 256, 0, s>>>(L.nn, L.agg.p, Phat.rowptr.p, Phat.col.p));
  AMGC_LAUNCH(k_tentative_qr<<<div_up((int64_t)n_agg * 32, 128), 128, 0, s>>>(n_agg, L.bu, mptr.p, midx.p, L.B.p, Phat.val.p, C.B.p,
                                                                  h->status.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(check_status(h, "tentative prolongator"));
  // --- multiplier tentative transfer
  AMGC_TRY(bucket_lists(L.nl, L.lagg.p, n_lagg, L.rl_ptr, L.rl_idx, s));
  AMGC_TRY(C.Bl.alloc(std::max(n_lagg, 1)));
  AMGC_TRY(L.pl_w.alloc(std::max(L.nl, 1)));
  DBsr Pl, Rl;
  if (L.nl > 0) {
    AMGC_LAUNCH(k_lm_norm<<<div_up(n_lagg, 128), 128, 0, s>>>(n_lagg, L.rl_ptr.p, L.rl_idx.p, L.Bl.p, C.Bl.p));
    AMGC_LAUNCH(k_lm_weight<<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.lagg.p, L.Bl.p, C.Bl.p, L.pl_w.p));
    Pl.nbr = L.nl; Pl.nbc = n_lagg; Pl.br = 3; Pl.bc = 3; Pl.nnzb = L.nl;
    AMGC_TRY(Pl.rowptr.alloc(L.nl + 1));
    AMGC_TRY(Pl.col.alloc(L.nl));
    AMGC_TRY(Pl.val.alloc((size_t)L.nl * 9));
    AMGC_LAUNCH(k_pl_bsr<<<div_up(L.nl + 1, 128), 128, 0, s>>>(L.nl, L.lagg.p, L.pl_w.p, Pl.rowptr.p, Pl.col.p, Pl.val.p));
    Rl.nbr = n_lagg; Rl.nbc = L.nl; Rl.br = 3; Rl.bc = 3; Rl.nnzb = L.nl;
    AMGC_TRY(Rl.rowptr.alloc(n_lagg + 1));
    AMGC_TRY(Rl.col.alloc(L.nl));
    AMGC_TRY(Rl.val.alloc((size_t)L.nl * 9));
    AMGC_LAUNCH(k_rl_bsr<<<div_up(n_lagg + 1, 128), 128, 0, s>>>(n_lagg, L.rl_ptr.p, L.rl_idx.p, L.pl_w.p, Rl.rowptr.p, Rl.col.p,
                                                      Rl.val.p));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  ptm.reset();
  // --- lambda_max and smoothed prolongator
  ptm.reset(new PhaseTimer(h, 5));
  if (L.kdiag.p == nullptr) AMGC_TRY(smoother_setup(h, l));
  AMGC_TRY(smoother_finish(h, l));
  if (h->opts.transfer == 1) {
    AMGC_TRY(spgemm(h, L.K, Phat, L.P));
    const double omega = h->opts.sa_omega / L.lam_max;
    DBuf<double> wdof;   // per-DOF SA damping of a batched level (sa_omega / lambda_max of the instance)
    if (h->n_inst > 1) {
      std::vector<double> w(L.nu());
      for (int q = 0; q < h->n_inst; ++q)
        for (int i = L.bu * L.nptr[q]; i < L.bu * L.nptr[q + 1]; ++i) w[i] = h->opts.sa_omega / L.inst_lam_max[q];
      AMGC_TRY(wdof.alloc(L.nu()));
      AMGC_CUDA_TRY(cudaMemcpyAsync(wdof.p, w.data(), L.nu() * sizeof(double), cudaMemcpyHostToDevice, s));
      AMGC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (L.bu == 3)
      AMGC_LAUNCH(k_sa_values<3><<<div_up((int64_t)L.nn * 32, 128), 128, 0, s>>>(L.nn, L.P.rowptr.p, L.P.col.p, L.agg.p, Phat.val.p, L.dinv.p,
                                                       omega, wdof.p, L.P.val.p));
    else
      AMGC_LAUNCH(k_sa_values<6><<<div_up((int64_t)L.nn * 32, 128), 128, 0, s>>>(L.nn, L.P.rowptr.p, L.P.col.p, L.agg.p, Phat.val.p, L.dinv.p,
                                                       omega, wdof.p, L.P.val.p));
    AMGC_CUDA_TRY(cudaGetLastError());
  } else {
    L.P = std::move(Phat);
  }
  ptm.reset();
  {
    PhaseTimer pt(h, 6);
    AMGC_TRY(bsr_transpose(h, L.P, L.R));
  }
  // --- Galerkin products
  ptm.reset(new PhaseTimer(h, 7));
  {
    DBsr AP;
    AMGC_TRY(spgemm(h, L.K, L.P, AP));
    AMGC_TRY(spgemm(h, L.R, AP, C.K, true));   // K_c = P^T K P is symmetric
  }
  if (L.nl > 0) {
    DBsr B1P, B2P;
    AMGC_TRY(spgemm(h, L.B1, Pl, B1P));
    AMGC_TRY(spgemm(h, L.R, B1P, C.B1));
    AMGC_TRY(spgemm(h, L.B2, L.P, B2P));
    AMGC_TRY(spgemm(h, Rl, B2P, C.B2));
    AMGC_TRY(C.Z.alloc((size_t)n_lagg * 9));
    AMGC_LAUNCH(k_zc<<<div_up(n_lagg, 128), 128, 0, s>>>(n_lagg, L.rl_ptr.p, L.rl_idx.p, L.pl_w.p, L.Z.p, C.Z.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    L.Pl = std::move(Pl);
    L.Rl = std::move(Rl);
  } else {
    C.B1.nbr = n_agg; C.B1.nbc = 0; C.B1.br = 6; C.B1.bc = 3;
    AMGC_TRY(C.B1.rowptr.alloc(n_agg + 1));
    AMGC_CUDA_TRY(cudaMemsetAsync(C.B1.rowptr.p, 0, (n_agg + 1) * sizeof(int), s));
    C.B2.nbr = 0; C.B2.nbc = n_agg; C.B2.br = 3; C.B2.bc = 6;
    AMGC_TRY(C.B2.rowptr.alloc(1));
    AMGC_CUDA_TRY(cudaMemsetAsync(C.B2.rowptr.p, 0, sizeof(int), s));
  }
  AMGC_TRY(check_status(h, "Galerkin products"));
  ptm.reset();
  // --- coarse per-node data
  AMGC_TRY(C.body.alloc(n_agg));   // body of a coarse node = body of its root (filled below)
  AMGC_TRY(C.lm_dnode.alloc(std::max(n_lagg, 1)));
  if (n_lagg > 0) AMGC_LAUNCH(k_copy_int<<<div_up(n_lagg, 256), 256, 0, s>>>(n_lagg, lm_dnode_c.p, C.lm_dnode.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  h->L.push_back(std::move(C));
  // (push_back may move the levels; re-fetch the references)
  Level& Lf = h->L[l];
  Level& Cn = h->L[l + 1];
  AMGC_LAUNCH(k_gather_body<<<div_up(n_agg, 256), 256, 0, s>>>(n_agg, roots.p, Lf.body.p, Cn.body.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

// ======================================================================== active-set update
// The constraint blocks B2 and Z are the only parts of the system that depend on the active set
// (inactive slave nodes: zero B2 row and -Z = I; active ones: the weighted-gap row and the
// tangential rows).  Aggregation, the transfers, lambda_max and the coarse K depend on K (and the
// interface pattern) alone, so an active-set change reuses them and forms anew: B2 and Z on the
// finest level, B2_c = R^lambda B2 P and Z_c on the coarser ones (B1_c does not change), the
// inverted Schur blocks (and their damping), the coarsest inverse (or the coarsest smoother data)
// and the FP32 mirrors.
int update_active_set(amgc_hierarchy* h, const uint8_t* active) {
  cudaStream_t s = h->stream;
  const int nlev = (int)h->L.size();
  Level& L0 = h->L[0];
  const int ns = L0.nl;
  DBuf<uint8_t> dAct;
  AMGC_TRY(dAct.alloc(std::max(ns, 1)));
  AMGC_CUDA_TRY(cudaMemcpyAsync(dAct.p, active, ns, cudaMemcpyDefault, s));
  // finest level: B2 (pattern and values) and Z
  DBsr B2;
  B2.nbr = ns; B2.nbc = L0.nn; B2.br = 3; B2.bc = 3;
  AMGC_TRY(B2.rowptr.alloc(ns + 1));
  AMGC_CUDA_TRY(cudaMemsetAsync(B2.rowptr.p, 0, (ns + 1) * sizeof(int), s));
  AMGC_LAUNCH(k_b2_count<<<div_up(ns, 256), 256, 0, s>>>(ns, dAct.p, L0.if_Mrp.p, B2.rowptr.p));
  int b2n = 0;
  AMGC_TRY(exclusive_scan(B2.rowptr.p, B2.rowptr.p, ns + 1, s, &b2n));
  B2.nnzb = b2n;
  AMGC_TRY(B2.col.alloc(std::max(b2n, 1)));
  AMGC_TRY(B2.val.alloc((size_t)std::max(b2n, 1) * 9));
  AMGC_LAUNCH(k_b2_fill<<<div_up(ns, 256), 256, 0, s>>>(ns, dAct.p, B2.rowptr.p, L0.if_Sl.p, L0.if_Ms.p, L0.if_D.p,
                                                       L0.if_Mrp.p, L0.if_Mcol.p, L0.if_Mv.p, L0.if_T.p, B2.col.p,
                                                       B2.val.p, L0.Z.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  L0.B2 = std::move(B2);
  L0.if_act = std::move(dAct);
  // coarser levels: B2_c = R^lambda (B2 P), Z_c = sum w^2 Z
  for (int l = 0; l + 1 < nlev; ++l) {
    Level& L = h->L[l];
    Level& C = h->L[l + 1];
    if (L.nl == 0) continue;
    DBsr B2P;
    AMGC_TRY(spgemm(h, L.B2, L.P, B2P));
    AMGC_TRY(spgemm(h, L.Rl, B2P, C.B2));
    AMGC_LAUNCH(k_zc<<<div_up(C.nl, 128), 128, 0, s>>>(C.nl, L.rl_ptr.p, L.rl_idx.p, L.pl_w.p, L.Z.p, C.Z.p));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  AMGC_TRY(check_status(h, "active-set update: constraint blocks"));
  // Schur blocks (and their damping) on every smoothed level, then the coarsest level
  const bool coarse_smooth = h->opts.coarse_solver == 1 && nlev > 1;
  for (int l = 0; l < nlev; ++l) {
    Level& L = h->L[l];
    const bool smoothed = l + 1 < nlev || coarse_smooth;
    if (!smoothed || L.nl == 0) continue;
    if (L.bu == 3)
      AMGC_LAUNCH(k_schur<3><<<div_up((int64_t)L.nl * 32, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p,
                                                   L.B1.rowptr.p, L.B1.col.p, L.B1.val.p, L.atinv.p, L.Z.p, L.Sinv.p,
                                                   h->status.p));
    else
      AMGC_LAUNCH(k_schur<6><<<div_up((int64_t)L.nl * 32, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p,
                                                   L.B1.rowptr.p, L.B1.col.p, L.B1.val.p, L.atinv.p, L.Z.p, L.Sinv.p,
                                                   h->status.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    AMGC_TRY(check_status(h, "active-set update: Schur blocks"));
    if (h->opts.schur_damping) AMGC_TRY(schur_damping_setup(h, L));
  }
  if (!coarse_smooth) AMGC_TRY(coarse_setup(h, nlev - 1));
  // transposed data is formed again on the next transposed call
  for (auto& L : h->L) {
    L.has_transposed = false;
    L.B1T = DBsr();
    L.B2T = DBsr();
  }
  // statistics of the changed blocks
  amgc_stats_t& st = h->stats;
  double nnz0 = 0.0, nnz_all = 0.0;
  for (int l = 0; l < nlev; ++l) {
    const Level& L = h->L[l];
    st.nnz[l] = L.K.nnzb * L.bu * L.bu + L.B1.nnzb * L.bu * 3 + L.B2.nnzb * 3 * L.bu + (int64_t)L.nl * 9;
    if (l == 0) nnz0 = (double)st.nnz[l];
    nnz_all += (double)st.nnz[l];
  }
  st.operator_complexity = nnz0 > 0 ? nnz_all / nnz0 : 0.0;
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

// ======================================================================== transposed-cycle data
__global__ void k_transpose3(int n, const double* __restrict__ a, double* __restrict__ t) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n) return;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) t[(int64_t)l * 9 + c * 3 + r] = a[(int64_t)l * 9 + r * 3 + c];
}
__global__ void k_transpose_dense(int n, const double* __restrict__ a, double* __restrict__ t) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  t[(int64_t)j * n + i] = a[idx];
}

// Builds, once, what the transposed V-cycle needs on every level.
int transposed_setup(amgc_hierarchy* h) {
  cudaStream_t s = h->stream;
  const int nlev = (int)h->L.size();
  for (int l = 0; l < nlev; ++l) {
    Level& L = h->L[l];
    if (L.has_transposed) continue;
    AMGC_TRY(bsr_transpose(h, L.B1, L.B1T));
    AMGC_TRY(bsr_transpose(h, L.B2, L.B2T));
    AMGC_TRY(L.ZT.alloc((size_t)std::max(L.nl, 1) * 9));
    if (L.nl > 0) AMGC_LAUNCH(k_transpose3<<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.Z.p, L.ZT.p));
    if (l < nlev - 1) {
      AMGC_TRY(L.SinvT.alloc((size_t)std::max(L.nl, 1) * 9));
      if (L.nl > 0) AMGC_LAUNCH(k_transpose3<<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.Sinv.p, L.SinvT.p));
      DBuf<int> flag;
      AMGC_TRY(flag.alloc(L.nn + 1));
      AMGC_LAUNCH(k_nonempty<<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B2T.rowptr.p, flag.p));
      int cnt = 0;
      AMGC_TRY(exclusive_scan(flag.p, flag.p, L.nn, s, &cnt));
      L.n_b2t_rows = cnt;
      if (h->opts.jacobi_sweeps > 1) AMGC_TRY(L.tsw.alloc((size_t)2 * std::max(L.nu(), 1)));
      AMGC_TRY(L.b2t_rows.alloc(std::max(cnt, 1)));
      AMGC_LAUNCH(k_compact<<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B2T.rowptr.p, flag.p, L.b2t_rows.p));
    } else {
      const int n = L.rows();
      AMGC_TRY(L.AinvT.alloc((size_t)n * n));
      AMGC_LAUNCH(k_transpose_dense<<<div_up((int64_t)n * n, 256), 256, 0, s>>>(n, L.Ainv.p, L.AinvT.p));
    }
    AMGC_CUDA_TRY(cudaGetLastError());
    L.has_transposed = true;
  }
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return make_views(h);
}

// ======================================================================== coarsest level: dense inverse
// dense copy of a BSR matrix into rows row0.., columns col0.. of A (row-major, n columns); one
// warp per block row, the lanes over the row's values
template <int BR, int BC>
__global__ void k_dense_put(int nbr, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                            int row0, int col0, double sign, int n, double* __restrict__ A) {
  constexpr int NQ = BR * BC;
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (i >= nbr) return;
  const int e0 = rp[i], nq = (rp[i + 1] - e0) * NQ;
  for (int q = lane; q < nq; q += 32) {
    const int eb = q / NQ;
    const int w = q - eb * NQ;
    const int r = w / BC, c = w - r * BC;
    A[(int64_t)(row0 + i * BR + r) * n + col0 + col[e0 + eb] * BC + c] = sign * val[(int64_t)e0 * NQ + q];
  }
}
__global__ void k_dense_z(int nl, const double* __restrict__ Z, int off, int n, double* __restrict__ A) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[(int64_t)(off + 3 * l + r) * n + off + 3 * l + c] = -Z[(int64_t)l * 9 + r * 3 + c];
}
// Gauss-Jordan step k, single block: pivot search (largest |A[i][k]|, i >= k, ties to the
// smallest i), row swap, scaling of the pivot row, and the multiplier column f.
__global__ void k_gj_pivot(int n, int k, double* __restrict__ A, int* __restrict__ piv, double* __restrict__ f, int* st) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int besti = n;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double v = fabs(A[(int64_t)i * n + k]);
    if (v > best || (v == best && i < besti)) { best = v; besti = i; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v = bv[threadIdx.x + o];
      int ii = bi[threadIdx.x + o];
      if (v > bv[threadIdx.x] || (v == bv[threadIdx.x] && ii < bi[threadIdx.x])) {
        bv[threadIdx.x] = v;
        bi[threadIdx.x] = ii;
      }
    }
    __syncthreads();
  }
  const int p = bi[0];
  const double pmax = bv[0];
  if (threadIdx.x == 0) piv[k] = p;
  if (p != k && p < n) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double t = A[(int64_t)k * n + j];
      A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
      A[(int64_t)p * n + j] = t;
    }
  }
  __syncthreads();
  double pv = A[(int64_t)k * n + k];
  if (!(pmax > 0.0) || !isfinite(pv)) {
    if (threadIdx.x == 0) set_status(st, ST_SINGULAR);
    pv = 1.0;
  }
  __syncthreads();
  // multiplier column (taken before the pivot row is scaled; column k is then cleared)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    f[i] = (i == k) ? 0.0 : A[(int64_t)i * n + k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (i != k) A[(int64_t)i * n + k] = 0.0;
  if (threadIdx.x == 0) A[(int64_t)k * n + k] = 1.0;
  __syncthreads();
  const double inv = 1.0 / pv;
  for (int j = threadIdx.x; j < n; j += blockDim.x) A[(int64_t)k * n + j] *= inv;
}
__global__ void k_gj_update(int n, int k, double* __restrict__ A, const double* __restrict__ f) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (i == k) return;
  const double fi = f[i];
  if (fi != 0.0) A[idx] -= fi * A[(int64_t)k * n + j];
}
// undo the row interchanges: swap columns k and piv[k] for k = n-1 .. 0 (one thread per row)
__global__ void k_gj_unscramble(int n, const int* __restrict__ piv, double* __restrict__ A) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = A + (int64_t)i * n;
  for (int k = n - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k) {
      double t = row[k];
      row[k] = row[p];
      row[p] = t;
    }
  }
}

// Gauss-Jordan inverse with partial pivoting in one cooperative launch: every step is one
// grid-wide pass, separated by grid barriers, between two n x n buffers (cur -> nxt).  Step k:
// every CTA finds the same pivot p = argmax_{i >= k} |cur[i][k]| (ties to the smallest i), keeps
// rows p and k of cur in shared memory, and writes its own rows of nxt:
//   row k  = row p / pv, with pv^-1 in column k;
//   row p  = row k - row k[k] * (new row k), with -row k[k] / pv in column k (p != k);
//   row i  = row i - row i[k] * (new row k), with -row i[k] / pv in column k.
// This is the in-place elimination of the single-block kernels with the interchange applied to
// whole rows; afterwards the columns are permuted back (interchanges in reverse order) into the
// other buffer.  Reads of cur bypass L1 (other CTAs wrote it before the barrier).
constexpr int kGjcThreads = 256;
__global__ void __launch_bounds__(kGjcThreads)
k_gj_coop(int n, double* __restrict__ Aa, double* __restrict__ Ab, int* __restrict__ piv, int* st) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double gj_sh[];   // [0, n): row p of cur, [n, 2n): row k of cur
  __shared__ double bv[kGjcThreads];
  __shared__ int bi[kGjcThreads];
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = min(n, (int)blockIdx.x * per), r1 = min(n, r0 + per);
  double* cur = Aa;
  double* nxt = Ab;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int besti = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      const double v = fabs(__ldcg(cur + (int64_t)i * n + k));
      if (v > best || (v == best && i < besti)) { best = v; besti = i; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const double v = bv[threadIdx.x + o];
        const int ii = bi[threadIdx.x + o];
        if (v > bv[threadIdx.x] || (v == bv[threadIdx.x] && ii < bi[threadIdx.x])) {
          bv[threadIdx.x] = v;
          bi[threadIdx.x] = ii;
        }
      }
      __syncthreads();
    }
    const int p = bi[0] < n ? bi[0] : k;
    const double pmax = bv[0];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      gj_sh[j] = __ldcg(cur + (int64_t)p * n + j);
      gj_sh[n + j] = __ldcg(cur + (int64_t)k * n + j);
    }
    __syncthreads();
    double pv = gj_sh[k];
    if (!(pmax > 0.0) || !isfinite(pv)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_status(st, ST_SINGULAR);
      pv = 1.0;
    }
    const double inv = 1.0 / pv;
    for (int i = r0; i < r1; ++i) {
      double* dst = nxt + (int64_t)i * n;
      if (i == k) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = j == k ? inv : gj_sh[j] * inv;
      } else {
        const double* src = i == p ? gj_sh + n : cur + (int64_t)i * n;
        const double a = i == p ? gj_sh[n + k] : __ldcg(src + k);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          const double v = i == p ? src[j] : __ldcg(src + j);
          dst[j] = j == k ? -a * inv : v - a * (gj_sh[j] * inv);
        }
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) piv[k] = p;
    grid.sync();
    double* t = cur;
    cur = nxt;
    nxt = t;
  }
  int* perm = reinterpret_cast<int*>(gj_sh);
  for (int j = threadIdx.x; j < n; j += blockDim.x) perm[j] = j;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = n - 1; k >= 0; --k) {
      const int p = __ldcg(piv + k);
      if (p != k) {
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
      }
    }
  }
  __syncthreads();
  for (int i = r0; i < r1; ++i)
    for (int j = threadIdx.x; j < n; j += blockDim.x) nxt[(int64_t)i * n + j] = __ldcg(cur + (int64_t)i * n + perm[j]);
}

// The same inverse with kGjB pivots per grid barrier (n up to kGjBlockedMax).  Per super-step
// every CTA (redundantly) eliminates the panel of columns K..K+b-1 in shared memory, recording
// the pivot rows' entities, the pivots and every row's multipliers a_e(t) (its panel value in
// column K+t just before step t).  The rows of the other columns then follow from the pivot rows
// of the super-step,
//   q_t = (row_{pi_t} - sum_{s<t} a_{pi_t}(s) q_s) / pv_t,
//   row_e <- row_e - sum_t a_e(t) q_t          (pivot row pi_s: q_s - sum_{t>s} a_{pi_s}(t) q_t),
// which is the per-column elimination with the same operations grouped per super-step.  Each CTA
// writes its own rows of the next buffer in the row order after the super-step's interchanges.
//
// GB300 issues FP64 at 2 FMA per clock and SM, so the redundant panel work is kept small: step t
// updates, for every row, only the columns right of t (what later pivot searches and
// multipliers read); column t of a row is left at its multiplier a_e(t).  The panel columns left
// of the pivot (the inverse's part) are formed only where they are needed, by replaying the
// step updates on the frozen multipliers: for the pivot row of each step (its scaled row is
// kept in ppan[t][.]) and, at the end of the super-step, for the CTA's own rows.  Every value
// is formed by the same operations, in the same order, as in the per-column elimination.  The
// pivot search compares magnitudes as integers (the bit patterns of non-negative doubles are
// ordered like their values), which keeps it off the FP64 pipe.
constexpr int kGjBlockedMax = 960;   // n limit of the blocked kernel (8 pivots per barrier)
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v)) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ void argmax_key(unsigned long long& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}
template <int kGjB>
__global__ void __launch_bounds__(kGjcThreads)
k_gj_blocked(int n, double* __restrict__ Aa, double* __restrict__ Ab, int* __restrict__ piv, int* st) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double gjb_sh[];
  double* panel = gjb_sh;                 // [kGjB][n] panel column c of entity e at c * n + e
  double* q = panel + n * kGjB;           // [kGjB][n] transformed pivot rows (columns outside the panel)
  int* p2e = reinterpret_cast<int*>(q + kGjB * n);   // [n] position -> entity
  int* estep = p2e + n;                   // [n] super-step pivot index of an entity, -1 otherwise
  __shared__ double ppan[kGjB][kGjB], pinv[kGjB];
  __shared__ unsigned long long wv[kGjcThreads / 32];
  __shared__ int pent[kGjB], wi[kGjcThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = min(n, (int)blockIdx.x * per), r1 = min(n, r0 + per);
  double* cur = Aa;
  double* nxt = Ab;
  for (int K = 0; K < n; K += kGjB) {
    const int nb = min(kGjB, n - K);
    for (int idx = tid; idx < n * nb; idx += kGjcThreads) {
      const int e = idx / nb, c = idx - e * nb;
      panel[c * n + e] = __ldcg(cur + (int64_t)e * n + K + c);
    }
    for (int e = tid; e < n; e += kGjcThreads) {
      p2e[e] = e;
      estep[e] = -1;
    }
    __syncthreads();
    for (int t = 0; t < nb; ++t) {
      const int k = K + t;
      const double* col_t = panel + t * n;
      unsigned long long bv = 0ULL;
      int bi = n;
      for (int i = k + tid; i < n; i += kGjcThreads) {
        const unsigned long long v = abs_key(col_t[p2e[i]]);
        if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
      }
      argmax_key(bv, bi);
      if (lane == 0) { wv[wid] = bv; wi[wid] = bi; }
      __syncthreads();
      if (wid == 0) {
        unsigned long long v = lane < kGjcThreads / 32 ? wv[lane] : 0ULL;
        int i = lane < kGjcThreads / 32 ? wi[lane] : n;
        argmax_key(v, i);   // every lane holds the winner
        const int p = i < n ? i : k;
        const int ep = p2e[p];
        const double pv = col_t[ep];
        const bool bad = !(fabs(pv) > 0.0) || !isfinite(pv);
        const double inv = 1.0 / (bad ? 1.0 : pv);
        // the pivot row scaled: columns left of t replayed from its multipliers, t itself the
        // reciprocal, columns right of t from the panel
        if (lane < t) {
          double f = -panel[lane * n + ep] * pinv[lane];
          for (int s2 = lane + 1; s2 < t; ++s2) f = fma(-panel[s2 * n + ep], ppan[s2][lane], f);
          ppan[t][lane] = f * inv;
        } else if (lane < nb) {
          ppan[t][lane] = lane == t ? inv : panel[lane * n + ep] * inv;
        }
        __syncwarp();   // every lane has read p2e before lane 0 interchanges
        if (lane == 0) {
          if (bad && blockIdx.x == 0) set_status(st, ST_SINGULAR);
          pent[t] = ep;
          pinv[t] = inv;
          estep[ep] = t;
          if (blockIdx.x == 0) piv[k] = p;
          // row interchange of positions k and p
          p2e[p] = p2e[k];
          p2e[k] = ep;
        }
      }
      __syncthreads();
      // columns right of t: every row but the pivot row takes a_e(t) times the pivot row off;
      // the pivot row becomes the scaled row
      const int ep = pent[t];
      if (t + 1 < nb) {
        for (int e = tid; e < n; e += kGjcThreads) {
          if (e == ep) {
            for (int c = t + 1; c < nb; ++c) panel[c * n + e] = ppan[t][c];
          } else {
            const double a = col_t[e];
            for (int c = t + 1; c < nb; ++c) panel[c * n + e] = fma(-a, ppan[t][c], panel[c * n + e]);
          }
        }
      }
      __syncthreads();
    }
    // transformed pivot rows outside the panel
    for (int j = tid; j < n; j += kGjcThreads) {
      if (j >= K && j < K + nb) continue;
      double orig[kGjB];   // the pivot rows' values in column j, loaded together
#pragma unroll
      for (int t = 0; t < kGjB; ++t) orig[t] = t < nb ? __ldcg(cur + (int64_t)pent[t] * n + j) : 0.0;
#pragma unroll
      for (int t = 0; t < kGjB; ++t) {
        if (t < nb) {
          const int ep = pent[t];
          double v = orig[t];
          for (int s2 = 0; s2 < t; ++s2) v -= panel[s2 * n + ep] * q[s2 * n + j];
          q[t * n + j] = v * pinv[t];
        }
      }
    }
    __syncthreads();
    for (int i = r0; i < r1; ++i) {
      const int e = p2e[i];
      const int se = estep[e];
      double* dst = nxt + (int64_t)i * n;
      for (int j = tid; j < n; j += kGjcThreads) {
        double v;
        if (j >= K && j < K + nb) {
          // panel column c: from the scaled pivot row (a pivot row, c <= its step) or from the
          // frozen multiplier a_e(c), then the later steps' updates
          const int c = j - K;
          int s0;
          if (se >= 0 && c <= se) {
            v = ppan[se][c];
            s0 = se + 1;
          } else {
            v = -panel[c * n + e] * pinv[c];
            s0 = c + 1;
          }
          for (int s2 = s0; s2 < nb; ++s2) v = fma(-panel[s2 * n + e], ppan[s2][c], v);
        } else if (se >= 0) {
          v = q[se * n + j];
          for (int t = se + 1; t < nb; ++t) v -= panel[t * n + e] * q[t * n + j];
        } else {
          v = __ldcg(cur + (int64_t)e * n + j);
          for (int t = 0; t < nb; ++t) v -= panel[t * n + e] * q[t * n + j];
        }
        dst[j] = v;
      }
    }
    grid.sync();
    double* tb = cur;
    cur = nxt;
    nxt = tb;
  }
  int* perm = p2e;
  for (int j = tid; j < n; j += kGjcThreads) perm[j] = j;
  __syncthreads();
  if (tid == 0) {
    for (int k = n - 1; k >= 0; --k) {
      const int p = __ldcg(piv + k);
      if (p != k) {
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
      }
    }
  }
  __syncthreads();
  for (int i = r0; i < r1; ++i)
    for (int j = tid; j < n; j += kGjcThreads) nxt[(int64_t)i * n + j] = __ldcg(cur + (int64_t)i * n + perm[j]);
}

// ---- batched coarsest level: one dense block per instance
template <int BR, int BC>
__global__ void k_dense_put_batched(int nbr, const int* __restrict__ rp, const int* __restrict__ col,
                                    const double* __restrict__ val, int row0, int col0, const int* __restrict__ inst,
                                    const int* __restrict__ loc, const int* __restrict__ goff,
                                    const int64_t* __restrict__ doff, double* __restrict__ A) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double* v = val + (int64_t)e * BR * BC;
    for (int r = 0; r < BR; ++r) {
      const int gr = row0 + i * BR + r;
      const int q = inst[gr];
      const int n = goff[q + 1] - goff[q];
      for (int c = 0; c < BC; ++c) {
        const int gc = col0 + col[e] * BC + c;
        A[doff[q] + (int64_t)loc[gr] * n + loc[gc]] = v[r * BC + c];
      }
    }
  }
}
__global__ void k_dense_z_batched(int nl, const double* __restrict__ Z, int off, const int* __restrict__ inst,
                                  const int* __restrict__ loc, const int* __restrict__ goff,
                                  const int64_t* __restrict__ doff, double* __restrict__ A) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nl) return;
  for (int r = 0; r < 3; ++r) {
    const int gr = off + 3 * l + r;
    const int q = inst[gr];
    const int n = goff[q + 1] - goff[q];
    for (int c = 0; c < 3; ++c) A[doff[q] + (int64_t)loc[gr] * n + loc[off + 3 * l + c]] = -Z[(int64_t)l * 9 + r * 3 + c];
  }
}
// Gauss-Jordan inverse with partial pivoting of every instance block, one CTA per block; the
// same elimination as the single-matrix path, with block barriers between the phases.
constexpr int kGjThreads = 512;
__global__ void __launch_bounds__(kGjThreads)
k_gj_batched(int n_inst, const int* __restrict__ goff, const int64_t* __restrict__ doff, double* __restrict__ Aall,
             double* __restrict__ fall, int* __restrict__ pivall, int* st) {
  __shared__ double bv[kGjThreads];
  __shared__ int bi[kGjThreads];
  const int q = blockIdx.x;
  if (q >= n_inst) return;
  const int n = goff[q + 1] - goff[q];
  double* A = Aall + doff[q];
  double* f = fall + goff[q];
  int* piv = pivall + goff[q];
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int besti = n;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
      double v = fabs(A[(int64_t)i * n + k]);
      if (v > best || (v == best && i < besti)) { best = v; besti = i; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        double v = bv[threadIdx.x + o];
        int ii = bi[threadIdx.x + o];
        if (v > bv[threadIdx.x] || (v == bv[threadIdx.x] && ii < bi[threadIdx.x])) {
          bv[threadIdx.x] = v;
          bi[threadIdx.x] = ii;
        }
      }
      __syncthreads();
    }
    const int p = bi[0];
    const double pmax = bv[0];
    __syncthreads();
    if (threadIdx.x == 0) piv[k] = p;
    if (p != k && p < n) {
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double t = A[(int64_t)k * n + j];
        A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
        A[(int64_t)p * n + j] = t;
      }
    }
    __syncthreads();
    double pv = A[(int64_t)k * n + k];
    if (!(pmax > 0.0) || !isfinite(pv)) {
      if (threadIdx.x == 0) set_status(st, ST_SINGULAR);
      pv = 1.0;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = (i == k) ? 0.0 : A[(int64_t)i * n + k];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) A[(int64_t)i * n + k] = 0.0;
    if (threadIdx.x == 0) A[(int64_t)k * n + k] = 1.0;
    __syncthreads();
    const double inv = 1.0 / pv;
    for (int j = threadIdx.x; j < n; j += blockDim.x) A[(int64_t)k * n + j] *= inv;
    __syncthreads();
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) {
      const int i = (int)(idx / n), j = (int)(idx % n);
      if (i != k && f[i] != 0.0) A[idx] -= f[i] * A[(int64_t)k * n + j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double* row = A + (int64_t)i * n;
    for (int k = n - 1; k >= 0; --k) {
      const int p = piv[k];
      if (p != k) {
        double t = row[k];
        row[k] = row[p];
        row[p] = t;
      }
    }
  }
}

static int coarse_setup_batched(amgc_hierarchy* h, int l) {
  cudaStream_t s = h->stream;
  Level& L = h->L[l];
  const int ni = h->n_inst;
  const int rows = L.rows();
  const int nu = L.nu();
  std::vector<int> inst(rows), loc(rows), glob(rows), goff(ni + 1, 0);
  std::vector<int64_t> doff(ni + 1, 0);
  int g = 0;
  for (int q = 0; q < ni; ++q) {
    goff[q] = g;
    int t = 0;
    for (int r = L.bu * L.nptr[q]; r < L.bu * L.nptr[q + 1]; ++r, ++t, ++g) {
      inst[r] = q; loc[r] = t; glob[g] = r;
    }
    for (int r = nu + 3 * L.lptr[q]; r < nu + 3 * L.lptr[q + 1]; ++r, ++t, ++g) {
      inst[r] = q; loc[r] = t; glob[g] = r;
    }
    doff[q + 1] = doff[q] + (int64_t)t * t;
  }
  goff[ni] = g;
  if (g != rows) {
    set_error("batched coarsest level: instance ranges do not cover the level");
    return AMGC_EINVAL;
  }
  AMGC_TRY(L.c_inst.alloc(rows));
  AMGC_TRY(L.c_loc.alloc(rows));
  AMGC_TRY(L.c_glob.alloc(rows));
  AMGC_TRY(L.c_goff.alloc(ni + 1));
  AMGC_TRY(L.c_doff.alloc(ni + 1));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.c_inst.p, inst.data(), rows * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.c_loc.p, loc.data(), rows * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.c_glob.p, glob.data(), rows * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.c_goff.p, goff.data(), (ni + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  AMGC_CUDA_TRY(cudaMemcpyAsync(L.c_doff.p, doff.data(), (ni + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  const int64_t tot = doff[ni];
  AMGC_TRY(L.Ainv.alloc((size_t)std::max<int64_t>(tot, 1)));
  AMGC_CUDA_TRY(cudaMemsetAsync(L.Ainv.p, 0, (size_t)tot * sizeof(double), s));
  const int* ci = L.c_inst.p;
  const int* cl = L.c_loc.p;
  const int* cg = L.c_goff.p;
  const int64_t* cd = L.c_doff.p;
  if (L.bu == 3) {
    AMGC_LAUNCH(k_dense_put_batched<3, 3><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p, 0,
                                                                           0, ci, cl, cg, cd, L.Ainv.p));
    if (L.nl > 0) {
      AMGC_LAUNCH(k_dense_put_batched<3, 3><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.B1.rowptr.p, L.B1.col.p,
                                                                             L.B1.val.p, 0, nu, ci, cl, cg, cd, L.Ainv.p));
      AMGC_LAUNCH(k_dense_put_batched<3, 3><<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p,
                                                                             L.B2.val.p, nu, 0, ci, cl, cg, cd, L.Ainv.p));
    }
  } else {
    AMGC_LAUNCH(k_dense_put_batched<6, 6><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p, 0,
                                                                           0, ci, cl, cg, cd, L.Ainv.p));
    if (L.nl > 0) {
      AMGC_LAUNCH(k_dense_put_batched<6, 3><<<div_up(L.nn, 128), 128, 0, s>>>(L.nn, L.B1.rowptr.p, L.B1.col.p,
                                                                             L.B1.val.p, 0, nu, ci, cl, cg, cd, L.Ainv.p));
      AMGC_LAUNCH(k_dense_put_batched<3, 6><<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p,
                                                                             L.B2.val.p, nu, 0, ci, cl, cg, cd, L.Ainv.p));
    }
  }
  if (L.nl > 0)
    AMGC_LAUNCH(k_dense_z_batched<<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.Z.p, nu, ci, cl, cg, cd, L.Ainv.p));
  DBuf<double> f;
  DBuf<int> piv;
  AMGC_TRY(f.alloc(std::max(rows, 1)));
  AMGC_TRY(piv.alloc(std::max(rows, 1)));
  AMGC_LAUNCH(k_gj_batched<<<ni, kGjThreads, 0, s>>>(ni, cg, cd, L.Ainv.p, f.p, piv.p, h->status.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(check_status(h, "batched coarsest factorisation"));
  AMGC_TRY(alloc_work(L));
  return AMGC_OK;
}

// In-place inverse of the dense row-major n x n matrix A by Gauss-Jordan elimination with partial
// pivoting (one cooperative launch where the device allows it, else a pivot and an update launch
// per column); a zero pivot sets ST_SINGULAR, which the caller's status check reports.
int dense_inverse(amgc_hierarchy* h, double* A, int n) {
  cudaStream_t s = h->stream;
  DBuf<int> piv;
  AMGC_TRY(piv.alloc(n));
  // one cooperative launch when the device supports it and two rows fit in shared memory,
  // else one pivot launch and one update launch per column
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  AMGC_CUDA_TRY(cudaGetDevice(&dev));
  AMGC_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  AMGC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // kGjB pivots per barrier while the panel tables fit in shared memory, else one per barrier
  const bool blocked = n <= kGjBlockedMax;
  const int gjb = 8;
  const void* kern = !blocked ? (const void*)k_gj_coop : (const void*)k_gj_blocked<8>;
  const size_t smem = blocked ? (size_t)n * (2 * gjb * sizeof(double) + 2 * sizeof(int))
                              : 2 * (size_t)n * sizeof(double);
  if (coop && smem <= 200 * 1024) {
    // (raised whatever the size: the kernel's static shared memory counts against 48 KB too)
    AMGC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AMGC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGjcThreads, smem));
  }
  if (per_sm > 0) {
    // the blocked kernel repeats the panel elimination in every CTA: one CTA per SM
    const int grid = std::min(n, blocked ? sms : sms * std::min(per_sm, 2));
    DBuf<double> tmp;
    AMGC_TRY(tmp.alloc((size_t)n * n));
    int nn = n;
    double* a = A;
    double* b = tmp.p;
    int* pv = piv.p;
    int* st = h->status.p;
    void* args[] = {&nn, &a, &b, &pv, &st};
    AMGC_CUDA_TRY(AMGC_LAUNCH(cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kGjcThreads), args, smem, s)));
    // the buffers alternate once per barrier; the permuted result is in the other one
    const int passes = blocked ? (n + gjb - 1) / gjb : n;
    if (passes % 2 == 0)
      AMGC_CUDA_TRY(cudaMemcpyAsync(A, tmp.p, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    DBuf<double> f;
    AMGC_TRY(f.alloc(n));
    const int64_t nn2 = (int64_t)n * n;
    for (int k = 0; k < n; ++k) {
      AMGC_LAUNCH(k_gj_pivot<<<1, 1024, 0, s>>>(n, k, A, piv.p, f.p, h->status.p));
      AMGC_LAUNCH(k_gj_update<<<div_up(nn2, 256), 256, 0, s>>>(n, k, A, f.p));
    }
    AMGC_LAUNCH(k_gj_unscramble<<<div_up(n, 128), 128, 0, s>>>(n, piv.p, A));
    AMGC_CUDA_TRY(cudaGetLastError());
  }
  return AMGC_OK;
}

int coarse_setup(amgc_hierarchy* h, int l) {
  if (h->n_inst > 1) return coarse_setup_batched(h, l);
  cudaStream_t s = h->stream;
  Level& L = h->L[l];
  const int n = L.rows();
  const int nu = L.nu();
  AMGC_TRY(L.Ainv.alloc((size_t)n * n));
  AMGC_CUDA_TRY(cudaMemsetAsync(L.Ainv.p, 0, (size_t)n * n * sizeof(double), s));
  if (L.bu == 3) {
    AMGC_LAUNCH(k_dense_put<3, 3><<<div_up((int64_t)L.nn * 32, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p, 0, 0, 1.0, n, L.Ainv.p));
    if (L.nl > 0) {
      AMGC_LAUNCH(k_dense_put<3, 3><<<div_up((int64_t)L.nn * 32, 128), 128, 0, s>>>(L.nn, L.B1.rowptr.p, L.B1.col.p, L.B1.val.p, 0, nu, 1.0, n,
                                                          L.Ainv.p));
      AMGC_LAUNCH(k_dense_put<3, 3><<<div_up((int64_t)L.nl * 32, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, nu, 0, 1.0, n,
                                                          L.Ainv.p));
    }
  } else {
    AMGC_LAUNCH(k_dense_put<6, 6><<<div_up((int64_t)L.nn * 32, 128), 128, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, L.K.val.p, 0, 0, 1.0, n, L.Ainv.p));
    if (L.nl > 0) {
      AMGC_LAUNCH(k_dense_put<6, 3><<<div_up((int64_t)L.nn * 32, 128), 128, 0, s>>>(L.nn, L.B1.rowptr.p, L.B1.col.p, L.B1.val.p, 0, nu, 1.0, n,
                                                          L.Ainv.p));
      AMGC_LAUNCH(k_dense_put<3, 6><<<div_up((int64_t)L.nl * 32, 128), 128, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, L.B2.val.p, nu, 0, 1.0, n,
                                                          L.Ainv.p));
    }
  }
  if (L.nl > 0) AMGC_LAUNCH(k_dense_z<<<div_up(L.nl, 128), 128, 0, s>>>(L.nl, L.Z.p, nu, n, L.Ainv.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(dense_inverse(h, L.Ainv.p, n));
  AMGC_TRY(check_status(h, "coarsest factorisation"));
  AMGC_TRY(alloc_work(L));
  return AMGC_OK;
}

}  // namespace amgc
