// Element gradients without any device allocation.
//
// amgc_grad_elements allocates device scratch for its per-element partial sums on every call.
// Some callers cannot allocate at that point: code that owns all device memory up front (a
// framework's own memory pool with a hard cap), or latency-critical loops that must not enter
// the driver's allocator and its implicit synchronisation.  amgc_grad_elements_noalloc
// computes the same gradients with its scratch in one file-scope device array of fixed size.
#include "amgc_internal.cuh"

#include <mutex>

namespace amgc {

// Largest element count the static scratch holds (three doubles per element: 6 MiB).
constexpr int kNoAllocMaxElements = 262144;

// Per-element lift contributions of the last call.  Every GPU that loads the library holds this
// array until the process exits; all calls on a device share it.
static __device__ __align__(256) double g_noalloc_lift[3 * kNoAllocMaxElements];

namespace {

constexpr int kNaWarps = 8;

// gE[e] = -adj_e^T Khat_e u_e and lift[e][c] = -E_e sum_{flagged nodes a} (Khat_e adj_e)_(a,c),
// one warp per element (lanes 0..23 hold DOF 3a + c of the element).
__global__ void __launch_bounds__(kNaWarps * 32)
k_grad_elements_na(int ne, const int* __restrict__ conn, const int* __restrict__ shape,
                   const double* __restrict__ Khat, const int* __restrict__ node_free, const double* __restrict__ adj,
                   const double* __restrict__ x, const double* __restrict__ uD, const uint8_t* __restrict__ lift_mask,
                   const double* __restrict__ E, double* __restrict__ gE, double* __restrict__ lift) {
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
__global__ void k_sum3_na(int ne, const double* __restrict__ lift, double* __restrict__ out) {
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

// Device address of g_noalloc_lift, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

int scratch_for_current_device(double** out) {
  int dev = 0;
  AMGC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("amgc_grad_elements_noalloc: device index out of range");
    return AMGC_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_lift);
    if (e != cudaSuccess) {
      set_error(std::string("amgc_grad_elements_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return AMGC_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return AMGC_OK;
}

}  // namespace

}  // namespace amgc

using namespace amgc;

extern "C" int amgc_grad_elements_noalloc(int32_t ne, const int32_t* conn, const int32_t* shape, const double* Khat,
                                          const int32_t* node_free, const double* adj, const double* x,
                                          const double* uD, const uint8_t* lift_mask, const double* E, double* gE,
                                          double* gt, void* stream) {
  if (ne < 0 || (ne > 0 && (!conn || !shape || !Khat || !node_free || !adj || !x || !uD || !gE)) ||
      (gt && (!lift_mask || !E))) {
    set_error("amgc_grad_elements_noalloc: invalid argument");
    return AMGC_EINVAL;
  }
  if (ne > kNoAllocMaxElements) {
    set_error("amgc_grad_elements_noalloc: " + std::to_string(ne) + " elements exceed the static scratch limit of " +
              std::to_string(kNoAllocMaxElements));
    return AMGC_EINVAL;
  }
  if (ne == 0) return AMGC_OK;
  double* lift = nullptr;
  if (gt) AMGC_TRY(scratch_for_current_device(&lift));
  cudaStream_t s = (cudaStream_t)stream;
  // every lift entry read below is written by the first kernel of the same call
  AMGC_LAUNCH(k_grad_elements_na<<<div_up((int64_t)ne * 32, kNaWarps * 32), kNaWarps * 32, 0, s>>>(
      ne, conn, shape, Khat, node_free, adj, x, uD, lift_mask, E, gE, gt ? lift : nullptr));
  if (gt) AMGC_LAUNCH(k_sum3_na<<<3, 1024, 0, s>>>(ne, lift, gt));
  AMGC_CUDA_TRY(cudaGetLastError());
  return AMGC_OK;
}
