// scan.cu -- device-wide exclusive prefix sums: int32 -> int32 (list sorts)
// and int32 -> int64 (work offsets whose totals may pass 2^31).
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

template <class T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* total) {
  __shared__ T warp_tot[kThreads / kWarp];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T t = warp_tot[lane];
    T s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_tot[lane] = s - t;  // exclusive offsets of the warps
    if (lane == 31) *total = s;
  }
  __syncthreads();
  return x - v + warp_tot[wid];
}

template <class TI, class T>
__global__ void __launch_bounds__(kThreads) k_block_totals(const TI* __restrict__ in, int n,
                                                           T* __restrict__ totals) {
  __shared__ T tot;
  const long base = (long)blockIdx.x * kPerBlock + threadIdx.x * kItems;
  T s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k)
    if (base + k < n) s += in[base + k];
  block_exclusive_sum(s, &tot);
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

template <class TI, class T>
__global__ void __launch_bounds__(kThreads) k_block_scan(const TI* __restrict__ in, int n,
                                                         const T* __restrict__ offsets,
                                                         T* __restrict__ out) {
  __shared__ T tot;
  const long base = (long)blockIdx.x * kPerBlock + threadIdx.x * kItems;
  T v[kItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  T run = block_exclusive_sum(s, &tot) + (offsets ? offsets[blockIdx.x] : T(0));
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
    if (base + k == n - 1) out[n] = run;
  }
}

}  // namespace

template <class TI, class T>
static cudaError_t scan_rec(const TI* in, T* out, int n, T* tmp, cudaStream_t s, long long* launches) {
  const int nb = (n + kPerBlock - 1) / kPerBlock;
  if (nb <= 1) {
    k_block_scan<TI, T><<<1, kThreads, 0, s>>>(in, n, nullptr, out);
    ++*launches;
    return cudaGetLastError();
  }
  T* totals = tmp;
  T* offsets = tmp + nb;
  k_block_totals<TI, T><<<nb, kThreads, 0, s>>>(in, n, totals);
  ++*launches;
  cudaError_t e = scan_rec<T, T>(totals, offsets, nb, tmp + 2 * (size_t)nb + 1, s, launches);
  if (e != cudaSuccess) return e;
  k_block_scan<TI, T><<<nb, kThreads, 0, s>>>(in, n, offsets, out);
  ++*launches;
  return cudaGetLastError();
}

template <class TI, class T>
static cudaError_t scan_any(const TI* in, T* out, int n, DevBuf& tmp, cudaStream_t s, long long* launches) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(T), s);
  // scratch for all recursion levels: < 3 n / 4096 + 3 per level
  size_t need = 0;
  for (long m = n; m > kPerBlock; m = (m + kPerBlock - 1) / kPerBlock)
    need += 2 * ((m + kPerBlock - 1) / kPerBlock) + 1;
  cudaError_t e = tmp.ensure((need + 16) * sizeof(T));
  if (e != cudaSuccess) return e;
  return scan_rec<TI, T>(in, out, n, tmp.as<T>(), s, launches);
}

cudaError_t scan_exclusive(const int* in, int* out, int n, DevBuf& tmp, cudaStream_t s,
                           long long* launches) {
  return scan_any<int, int>(in, out, n, tmp, s, launches);
}

cudaError_t scan_exclusive64(const int* in, long long* out, int n, DevBuf& tmp, cudaStream_t s,
                             long long* launches) {
  return scan_any<int, long long>(in, out, n, tmp, s, launches);
}

}  // namespace dfgt
