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

// Device address of g_noalloc_lift, looked up once per device (with that device current).  A
// cudaDeviceReset unloads the module and makes the cached address stale: the library is not to be
// used on a device after a reset in the same process (the header says so).
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
  // the kernels of amgc_grad_elements, with the static array as their scratch; no synchronisation
  return launch_grad_elements(ne, conn, shape, Khat, node_free, adj, x, uD, lift_mask, E, gE, gt, lift,
                              (cudaStream_t)stream);
}
