// tcgen05_accum_probe.cu -- test helper (built and run by
// test_gpu_tcgen05_model.py): checks the operand layout the tensor-core
// exact sums use (tcgen05.mma kind::f16, M = N = 128, float16 A and B
// K-major without swizzle in 8-row x 16-byte core matrices, 2048 bytes
// between K groups of 8 and 128 bytes between 8-row groups, float32 D in
// tensor memory read back with tcgen05.ld 32x32b) element by element
// against float64 sums, and measures the accumulation error over K16
// steps in units of 2^-24 of the sum of |products|, for random operands
// and for operands whose second K half cancels the first.
#include <cstdint>
#include <cstdio>
#include <cuda_fp16.h>

__device__ unsigned hash(unsigned x) {
  x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
  return x;
}
__device__ float urand(unsigned s) { return (hash(s) >> 8) * (1.0f / 16777216.0f); }
// random sign, magnitude 2^[-6, 6) with a random mantissa
__device__ float rv(unsigned s) {
  const float m = 1.f + urand(s * 3 + 1);
  const int e = (int)(urand(s * 3 + 2) * 12.f) - 6;
  return ldexpf(m, e) * (urand(s * 3 + 3) < 0.5f ? -1.f : 1.f);
}

constexpr int kRows = 128;
constexpr int kMaxK = 112;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(2048 >> 4) << 16) | ((uint64_t)(128 >> 4) << 32) |
         ((uint64_t)1 << 46);
}
// half index of element (row, k) of a 128-row K-major tile
__device__ __forceinline__ int at(int row, int k) { return ((k >> 3) * 16 + (row >> 3)) * 64 + (row & 7) * 8 + (k & 7); }

__global__ void __launch_bounds__(128) probe(int K, int mode, double* worst, int* bad, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __half* A = reinterpret_cast<__half*>(smem);
  __half* B = reinterpret_cast<__half*>(smem + kRows * kMaxK * 2);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned base = (blockIdx.x * 4 + mode) * 131072u + K;
  for (int i = tid; i < kRows * K; i += 128) {
    const int r = i / K, k = i % K;
    float a = rv(base + i), b = rv(base + 50000 + i);
    if (mode == 1 && k >= K / 2) {  // the second half cancels the first up to rounding
      a = rv(base + r * K + (k - K / 2));
      b = -rv(base + 50000 + r * K + (k - K / 2)) * (1.f + 0.01f * (urand(base + 90000 + i) - 0.5f));
    }
    A[at(r, k)] = __float2half_rn(a);
    B[at(r, k)] = __float2half_rn(b);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | ((uint32_t)(kRows >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
  if (tid == 0) {
    for (int ks = 0; ks < K / 16; ++ks) {
      const uint64_t ad = desc(saddr(A) + ks * 4096), bd = desc(saddr(B) + ks * 4096);
      const uint32_t acc = ks > 0;
      asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                       tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&mbar)));
  }
  uint32_t done = 0;
  for (int it = 0; it < (1 << 22) && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(saddr(&mbar)), "r"(0u) : "memory");
  const bool ok = __all_sync(0xffffffffu, done != 0);
  if (!ok && lane == 0) atomicOr(status, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = warp * 32 + lane;
  for (int c0 = 0; ok && c0 < kRows; c0 += 32) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(tmem + ((uint32_t)(warp * 32) << 16) + c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    for (int j = 0; j < 32; ++j) {
      const int col = c0 + j;
      double s = 0, sa = 0;
      for (int k = 0; k < K; ++k) {
        const double p = (double)__half2float(A[at(row, k)]) * (double)__half2float(B[at(col, k)]);
        s += p;
        sa += fabs(p);
      }
      const double err = fabs((double)__uint_as_float(r[j]) - s) / (sa > 0 ? sa : 1.0) * 16777216.0;
      if (err > 64.0) atomicAdd(bad, 1);
      unsigned long long* wp = reinterpret_cast<unsigned long long*>(worst) + mode;
      unsigned long long v = __double_as_longlong(err), o = *wp;
      while (v > o) {
        const unsigned long long p2 = atomicCAS(wp, o, v);
        if (p2 == o) break;
        o = p2;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

int main() {
  double* w;
  int *bad, *st;
  cudaMalloc(&w, 2 * sizeof(double));
  cudaMalloc(&bad, sizeof(int));
  cudaMalloc(&st, sizeof(int));
  const int smem = 2 * kRows * kMaxK * 2;
  cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int Ks[3] = {32, 64, 112};
  for (int K : Ks) {
    cudaMemset(w, 0, 2 * sizeof(double));
    cudaMemset(bad, 0, sizeof(int));
    cudaMemset(st, 0, sizeof(int));
    for (int mode = 0; mode < 2; ++mode) probe<<<96, 128, smem>>>(K, mode, w, bad, st);
    const cudaError_t e = cudaDeviceSynchronize();
    double hw[2] = {0, 0};
    int hb = 0, hs = 0;
    cudaMemcpy(hw, w, sizeof hw, cudaMemcpyDeviceToHost);
    cudaMemcpy(&hb, bad, sizeof hb, cudaMemcpyDeviceToHost);
    cudaMemcpy(&hs, st, sizeof hs, cudaMemcpyDeviceToHost);
    printf("K=%d status=%d wait=%d worst_random=%.4f worst_cancel=%.4f off=%d steps=%d\n", K, (int)e, hs, hw[0], hw[1],
           hb, K / 16);
    if (e != cudaSuccess) return 1;
  }
  return 0;
}
