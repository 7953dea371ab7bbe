// Active-set changes of the frictionless contact problem: the setup reuse of an existing hierarchy
// (the constraint blocks formed anew, everything K determines kept) and the primal-dual active set
// strategy (PDASS, Sec. 2.2) driving it.
//
// The discrete contact conditions (Eqs. ch4_discretenormalcontact, ch4_discretefrictionless) ask,
// at every slave node j, for a weighted gap g_j >= 0, a normal multiplier lambda_n,j >= 0 with
// g_j lambda_n,j = 0 and no tangential multiplier.  PDASS solves the linear saddle system of the
// current set (active: the normal row g_j(u) = 0 and the tangential rows; inactive: lambda_j = 0)
// and takes as next set the nodes with lambda_n,j - c g_j(u) > 0, until the set repeats.  With a
// geometric initial normal gap g0_j the weighted gap of the displaced configuration is
//     g_j(u) = D_jj g0_j - n_j^T (D_jj u_s,j - sum_l M_jl u_m,l),
// so an active node's normal row of B2 carries the right-hand side D_jj g0_j.
#include "amgc_internal.cuh"

#include <cmath>

namespace amgc {

// rhs = [f; g]: g_j = (D_jj g0_j, 0, 0) on active nodes (normal row, Cartesian multipliers in the
// triad's frame through B2 and Z), 0 on inactive ones
__global__ void k_pdass_rhs(int64_t nu, int ns, const double* __restrict__ f, const uint8_t* __restrict__ active,
                            const double* __restrict__ D, const double* __restrict__ g0, double* __restrict__ rhs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nu) rhs[i] = f[i];
  if (i < ns) {
    double* g = rhs + nu + 3 * i;
    g[0] = active[i] ? D[i] * g0[i] : 0.0;
    g[1] = 0.0;
    g[2] = 0.0;
  }
}

// next_j = [lambda_n,j - c g_j(u) > 0]; counts the nodes whose status changes
__global__ void k_pdass_next(int ns, const double* __restrict__ x, int64_t nu, const double* __restrict__ D,
                             const double* __restrict__ g0, const int* __restrict__ mrp, const int* __restrict__ mcol,
                             const double* __restrict__ mval, const int* __restrict__ slave_node,
                             const int* __restrict__ master_node, const double* __restrict__ triad, double c,
                             const uint8_t* __restrict__ active, uint8_t* __restrict__ next, int* __restrict__ changed) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ns) return;
  const double* n = triad + 9 * (int64_t)j;     // row 0 of the triad: the normal
  const double* us = x + 3 * (int64_t)slave_node[j];
  double v0 = D[j] * us[0], v1 = D[j] * us[1], v2 = D[j] * us[2];
  for (int q = mrp[j]; q < mrp[j + 1]; ++q) {
    const double* um = x + 3 * (int64_t)master_node[mcol[q]];
    v0 -= mval[q] * um[0];
    v1 -= mval[q] * um[1];
    v2 -= mval[q] * um[2];
  }
  const double gap = D[j] * g0[j] - (n[0] * v0 + n[1] * v1 + n[2] * v2);
  const double* lam = x + nu + 3 * (int64_t)j;
  const double lam_n = n[0] * lam[0] + n[1] * lam[1] + n[2] * lam[2];
  const uint8_t a = lam_n - c * gap > 0.0 ? 1 : 0;
  next[j] = a;
  if (a != active[j]) atomicAdd(changed, 1);
}

static int refresh_after_update(amgc_hierarchy* h) {
  drop_cycle_graphs(h);
  AMGC_TRY(make_views(h));
  // the nested preconditioner's exact Schur complement depends on the active set too
  if (!h->nest.empty()) AMGC_TRY(nested_setup(h));
  // and so do the block smoothers' Schur factors
  if (h->smoother_kind != 0) AMGC_TRY(block_smoother_setup(h, true));
  return AMGC_OK;
}

}  // namespace amgc

using namespace amgc;

extern "C" {

int amgc_update_active_set(struct amgc_hierarchy* h, const uint8_t* active, void* stream) {
  if (!h || !active) {
    set_error("amgc_update_active_set: invalid argument");
    return AMGC_EINVAL;
  }
  if (h->n_inst > 1) {
    set_error("amgc_update_active_set: not available for batched hierarchies");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  AMGC_TRY(update_active_set(h, active));
  return refresh_after_update(h);
}

int amgc_pdass(struct amgc_hierarchy* h, const double* f, const double* g0, double c, int32_t max_steps, double* x,
               uint8_t* active_out, int32_t* steps, int32_t* total_iters, void* stream) {
  if (steps) *steps = 0;
  if (total_iters) *total_iters = 0;
  if (!h || !f || !g0 || !x || !(c > 0.0) || !std::isfinite(c) || max_steps < 1) {
    set_error("amgc_pdass: invalid argument");
    return AMGC_EINVAL;
  }
  if (h->n_inst > 1) {
    set_error("amgc_pdass: not available for batched hierarchies");
    return AMGC_EINVAL;
  }
  h->stream = (cudaStream_t)stream;
  StreamScope scope_(h->stream);
  cudaStream_t s = h->stream;
  Level& L0 = h->L[0];
  const int ns = L0.nl;
  const int64_t nu = L0.nu();
  const int64_t n = L0.rows();
  DBuf<double> rhs;
  DBuf<uint8_t> next;
  DBuf<int> changed;
  AMGC_TRY(rhs.alloc(n));
  AMGC_TRY(next.alloc(std::max(ns, 1)));
  AMGC_TRY(changed.alloc(1));
  int it_sum = 0;
  for (int step = 0; step < max_steps; ++step) {
    Level& F = h->L[0];
    AMGC_LAUNCH(k_pdass_rhs<<<div_up(std::max<int64_t>(nu, ns), 256), 256, 0, s>>>(nu, ns, f, F.if_act.p, F.if_D.p, g0,
                                                                                  rhs.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    int it = 0;
    double rr = 0.0;
    const int st = fgmres(h, rhs.p, x, 0.0, &it, &rr);
    it_sum += it;
    if (steps) *steps = step + 1;
    if (total_iters) *total_iters = it_sum;
    if (st != AMGC_OK) return st;
    AMGC_CUDA_TRY(cudaMemsetAsync(changed.p, 0, sizeof(int), s));
    AMGC_LAUNCH(k_pdass_next<<<div_up(ns, 128), 128, 0, s>>>(ns, x, nu, F.if_D.p, g0, F.if_Mrp.p, F.if_Mcol.p, F.if_Mv.p,
                                                            F.if_Sl.p, F.if_Ms.p, F.if_T.p, c, F.if_act.p, next.p,
                                                            changed.p));
    AMGC_CUDA_TRY(cudaGetLastError());
    int nchg = 0;
    AMGC_CUDA_TRY(cudaMemcpyAsync(&nchg, changed.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
    if (nchg == 0) {
      if (active_out) {
        AMGC_CUDA_TRY(cudaMemcpyAsync(active_out, F.if_act.p, ns, cudaMemcpyDefault, s));
        AMGC_CUDA_TRY(cudaStreamSynchronize(s));
      }
      return AMGC_OK;
    }
    if (step + 1 == max_steps) break;      // no solve left for the next set: keep the last one
    AMGC_TRY(update_active_set(h, next.p));
    AMGC_TRY(refresh_after_update(h));
  }
  if (active_out) {
    AMGC_CUDA_TRY(cudaMemcpyAsync(active_out, h->L[0].if_act.p, ns, cudaMemcpyDefault, s));
    AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  }
  set_error("amgc_pdass: the active set still changed after max_steps solves");
  return AMGC_NOT_CONVERGED;
}

}  // extern "C"
