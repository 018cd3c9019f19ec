// scan.cu -- device-wide exclusive prefix sum of int32 (used by the tree build).
//
// Three passes: per-block totals, a scan of the totals (recursively), and a
// per-block scan that adds the block offset.  Each block covers 4096
// elements (1024 threads x 4 consecutive items).
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kThreads = 1024;
constexpr int kItems = 4;
constexpr int kPerBlock = kThreads * kItems;

__device__ __forceinline__ int block_exclusive_sum(int v, int* total) {
  __shared__ int warp_tot[kThreads / kWarp];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = warp_tot[lane];
    int s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_tot[lane] = s - t;  // exclusive offsets of the warps
    if (lane == 31) *total = s;
  }
  __syncthreads();
  return x - v + warp_tot[wid];
}

__global__ void __launch_bounds__(kThreads) k_block_totals(const int* __restrict__ in, int n,
                                                           int* __restrict__ totals) {
  __shared__ int tot;
  const long base = (long)blockIdx.x * kPerBlock + threadIdx.x * kItems;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k)
    if (base + k < n) s += in[base + k];
  block_exclusive_sum(s, &tot);
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kThreads) k_block_scan(const int* __restrict__ in, int n,
                                                         const int* __restrict__ offsets,
                                                         int* __restrict__ out) {
  __shared__ int tot;
  const long base = (long)blockIdx.x * kPerBlock + threadIdx.x * kItems;
  int v[kItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int run = block_exclusive_sum(s, &tot) + (offsets ? offsets[blockIdx.x] : 0);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
    if (base + k == n - 1) out[n] = run;
  }
}

}  // namespace

static cudaError_t scan_rec(const int* in, int* out, int n, int* tmp, cudaStream_t s,
                            long long* launches) {
  const int nb = (n + kPerBlock - 1) / kPerBlock;
  if (nb <= 1) {
    k_block_scan<<<1, kThreads, 0, s>>>(in, n, nullptr, out);
    ++*launches;
    return cudaGetLastError();
  }
  int* totals = tmp;
  int* offsets = tmp + nb;
  k_block_totals<<<nb, kThreads, 0, s>>>(in, n, totals);
  ++*launches;
  cudaError_t e = scan_rec(totals, offsets, nb, tmp + 2 * (size_t)nb + 1, s, launches);
  if (e != cudaSuccess) return e;
  k_block_scan<<<nb, kThreads, 0, s>>>(in, n, offsets, out);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t scan_exclusive(const int* in, int* out, int n, DevBuf& tmp, cudaStream_t s,
                           long long* launches) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int), s);
  // scratch for all recursion levels: < 3 n / 4096 + 3 per level
  size_t need = 0;
  for (long m = n; m > kPerBlock; m = (m + kPerBlock - 1) / kPerBlock)
    need += 2 * ((m + kPerBlock - 1) / kPerBlock) + 1;
  cudaError_t e = tmp.ensure((need + 16) * sizeof(int));
  if (e != cudaSuccess) return e;
  return scan_rec(in, out, n, tmp.as<int>(), s, launches);
}

}  // namespace dfgt
