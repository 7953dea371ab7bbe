// Gradient kernels of the adjoint path: the outer-product scatter -adj (x) x onto the stored
// blocks of K, B1 and B2, and the element-level gradients with respect to the element moduli
// (K = sum_e E_e Khat_e) and a uniform prescribed displacement (f = -K_fD u_D).
#include "amgc_internal.cuh"

namespace amgc {

// g[blk] = -a[row(blk)] (x) v[col(blk)] for a BSR with BR x BC blocks, one thread per block row
template <int BR, int BC>
__global__ void k_outer_scatter(int nbr, const int* __restrict__ rp, const int* __restrict__ col,
                                const double* __restrict__ a, const double* __restrict__ v, double* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nbr) return;
  double ai[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) ai[r] = a[(int64_t)i * BR + r];
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double* vj = v + (int64_t)col[e] * BC;
    double* out = g + (int64_t)e * BR * BC;
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int c = 0; c < BC; ++c) out[r * BC + c] = -ai[r] * vj[c];
  }
}

int grad_scatter(amgc_hierarchy* h, const double* adj, const double* x, double* gK, double* gB1, double* gB2) {
  const Level& L = h->L[0];
  const int nu = L.nu();
  cudaStream_t s = h->stream;
  AMGC_LAUNCH(k_outer_scatter<3, 3><<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.K.rowptr.p, L.K.col.p, adj, x, gK));
  if (gB1 && L.nl > 0)
    AMGC_LAUNCH(k_outer_scatter<3, 3><<<div_up(L.nn, 256), 256, 0, s>>>(L.nn, L.B1.rowptr.p, L.B1.col.p, adj, x + nu,
                                                                        gB1));
  if (gB2 && L.nl > 0)
    AMGC_LAUNCH(k_outer_scatter<3, 3><<<div_up(L.nl, 256), 256, 0, s>>>(L.nl, L.B2.rowptr.p, L.B2.col.p, adj + nu, x,
                                                                        gB2));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

// One warp per element: lanes 0..23 hold the element DOF k = 3a + c.
constexpr int kGradWarps = 8;
__global__ void __launch_bounds__(kGradWarps * 32)
k_grad_elements(int ne, const int* __restrict__ conn, const int* __restrict__ shape, const double* __restrict__ Khat,
                const int* __restrict__ node_free, const double* __restrict__ adj, const double* __restrict__ x,
                const double* __restrict__ uD, const uint8_t* __restrict__ lift_mask, const double* __restrict__ E,
                double* __restrict__ gE, double* __restrict__ lift) {
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= ne) return;
  double ak = 0.0, uk = 0.0;
  int node = 0;
  if (lane < 24) {
    node = conn[(int64_t)e * 8 + lane / 3];
    const int c = lane % 3;
    const int f = node_free[node];
    if (f >= 0) {
      ak = adj[3 * (int64_t)f + c];
      uk = x[3 * (int64_t)f + c];
    } else {
      uk = uD[3 * (int64_t)node + c];
    }
  }
  const double* Kh = Khat + (int64_t)shape[e] * 576;
  double ku = 0.0, ka = 0.0;
  for (int j = 0; j < 24; ++j) {
    const double uj = __shfl_sync(0xffffffffu, uk, j);
    const double aj = __shfl_sync(0xffffffffu, ak, j);
    if (lane < 24) {
      const double kv = Kh[lane * 24 + j];
      ku = fma(kv, uj, ku);
      ka = fma(kv, aj, ka);
    }
  }
  const double ge = warp_sum(-ak * ku);
  if (lane == 0) gE[e] = ge;
  if (lift != nullptr) {
    const double contrib = (lane < 24 && lift_mask[node]) ? -E[e] * ka : 0.0;
    // per element and component: sum over the element's nodes a (lanes 3a + c)
    double l0 = (lane % 3 == 0) ? contrib : 0.0, l1 = (lane % 3 == 1) ? contrib : 0.0,
           l2 = (lane % 3 == 2) ? contrib : 0.0;
    l0 = warp_sum(l0);
    l1 = warp_sum(l1);
    l2 = warp_sum(l2);
    if (lane == 0) {
      lift[3 * (int64_t)e] = l0;
      lift[3 * (int64_t)e + 1] = l1;
      lift[3 * (int64_t)e + 2] = l2;
    }
  }
}

// out[c] = sum_e lift[e][c], one block per component, fixed order (deterministic)
__global__ void k_sum3(int ne, const double* __restrict__ lift, double* __restrict__ out) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) s += lift[3 * (int64_t)e + c];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[c] = v;
  }
}

int launch_grad_elements(int ne, const int* conn, const int* shape, const double* Khat, const int* node_free,
                         const double* adj, const double* x, const double* uD, const uint8_t* lift_mask,
                         const double* E, double* gE, double* gt, double* lift, cudaStream_t s) {
  if (ne == 0) return AMGC_OK;
  // every lift entry k_sum3 reads is written by k_grad_elements of the same call
  AMGC_LAUNCH(k_grad_elements<<<div_up((int64_t)ne * 32, kGradWarps * 32), kGradWarps * 32, 0, s>>>(
      ne, conn, shape, Khat, node_free, adj, x, uD, lift_mask, E, gE, gt ? lift : nullptr));
  if (gt) AMGC_LAUNCH(k_sum3<<<3, 1024, 0, s>>>(ne, lift, gt));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}

int grad_elements(int ne, const int* conn, const int* shape, const double* Khat, const int* node_free,
                  const double* adj, const double* x, const double* uD, const uint8_t* lift_mask, const double* E,
                  double* gE, double* gt, cudaStream_t s) {
  if (ne == 0) return AMGC_OK;
  DBuf<double> lift;
  if (gt) AMGC_TRY(lift.alloc((size_t)ne * 3));
  AMGC_TRY(launch_grad_elements(ne, conn, shape, Khat, node_free, adj, x, uD, lift_mask, E, gE, gt, lift.p, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));   // lift is freed on return
  return AMGC_OK;
}

}  // namespace amgc
