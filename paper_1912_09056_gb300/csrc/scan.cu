// Exclusive prefix sum over int32 (row pointers, ranks, compaction offsets).
#include "amgc_internal.cuh"

namespace amgc {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void scan_tiles(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ tile_sums, int n) {
  __shared__ int warp_tot[kScanThreads / 32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int v[kScanItems];
  int run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = base + k;
    v[k] = idx < n ? in[idx] : 0;
    run += v[k];
  }
  // inclusive scan of per-thread totals within the warp
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;   // exclusive warp offsets
    if (lane == kScanThreads / 32 - 1 && tile_sums) tile_sums[blockIdx.x] = wi;
  }
  __syncthreads();
  int off = warp_tot[wid] + inc - run;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int idx = base + k;
    if (idx < n) out[idx] = off;
    off += v[k];
  }
}

__global__ void add_tile_offsets(int* __restrict__ out, const int* __restrict__ offs, int n) {
  int idx = blockIdx.x * kScanTile + threadIdx.x;
  int o = offs[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, idx += kScanThreads)
    if (idx < n) out[idx] += o;
}

int scan_rec(const int* in, int* out, int n, cudaStream_t s) {
  if (n <= 0) return AMGC_OK;
  int tiles = div_up(n, kScanTile);
  if (tiles == 1) {
    AMGC_LAUNCH(scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, nullptr, n));
    AMGC_CUDA_TRY(cudaGetLastError());
    return AMGC_OK;
  }
  DBuf<int> sums, offs;
  AMGC_TRY(sums.alloc(tiles));
  AMGC_TRY(offs.alloc(tiles));
  AMGC_LAUNCH(scan_tiles<<<tiles, kScanThreads, 0, s>>>(in, out, sums.p, n));
  AMGC_CUDA_TRY(cudaGetLastError());
  AMGC_TRY(scan_rec(sums.p, offs.p, tiles, s));
  AMGC_LAUNCH(add_tile_offsets<<<tiles, kScanThreads, 0, s>>>(out, offs.p, n));
  AMGC_CUDA_TRY(cudaGetLastError());
  // sums / offs go back to the pool on return, ordered on the allocation stream: wait only if the
  // scan ran on another stream
  if (!allocations_ordered_on(s)) AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  return AMGC_OK;
}

__global__ void k_scan_total(const int* __restrict__ last_out, int* __restrict__ t) {
  if (blockIdx.x == 0 && threadIdx.x == 0) t[1] = last_out[0] + t[0];
}

}  // namespace

// out[i] = sum_{k<i} in[k]; *total_host (optional) = sum of all inputs.  in may equal out.
// The total is formed on the device (the last input is saved before the scan, since in may equal
// out) and read back with one synchronisation.
int exclusive_scan(const int* in, int* out, int n, cudaStream_t s, int* total_host) {
  if (!total_host) return scan_rec(in, out, n, s);
  if (n <= 0) {
    *total_host = 0;
    return AMGC_OK;
  }
  DBuf<int> t;
  AMGC_TRY(t.alloc(2));
  AMGC_CUDA_TRY(cudaMemcpyAsync(t.p, in + n - 1, sizeof(int), cudaMemcpyDeviceToDevice, s));
  AMGC_TRY(scan_rec(in, out, n, s));
  AMGC_LAUNCH(k_scan_total<<<1, 32, 0, s>>>(out + n - 1, t.p));
  AMGC_CUDA_TRY(cudaGetLastError());
  int tot = 0;
  AMGC_CUDA_TRY(cudaMemcpyAsync(&tot, t.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMGC_CUDA_TRY(cudaStreamSynchronize(s));
  *total_host = tot;
  return AMGC_OK;
}

}  // namespace amgc
