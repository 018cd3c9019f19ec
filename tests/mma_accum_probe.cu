// mma_accum_probe.cu -- test helper (built and run by test_gpu_mma_model.py):
// checks the mma.sync fragment layouts the tensor-core exact sums use
// (m16n8k16 and m16n8k8, float16 operands, float32 C and D) element by
// element against float64 sums, and measures the accumulation error in
// units of 2^-24 of the sum of |terms| (C included) over random cases with
// C = 0, a C that cancels the products, and a random C.
#include <cstdio>
#include <cuda_fp16.h>
__device__ unsigned hash(unsigned x) { x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16; return x; }
__device__ float urand(unsigned s) { return (hash(s) >> 8) * (1.0f / 16777216.0f); }
// value: random sign, magnitude 2^[-6, 6) with random mantissa; some zero
__device__ __half rh(unsigned s) {
  float m = 1.f + urand(s * 3 + 1);
  int e = (int)(urand(s * 3 + 2) * 12.f) - 6;
  float v = ldexpf(m, e) * (urand(s * 3 + 3) < 0.5f ? -1.f : 1.f);
  return __float2half_rn(v);
}
__device__ unsigned pk(__half a, __half b) { return (unsigned)__half_as_ushort(a) | ((unsigned)__half_as_ushort(b) << 16); }
template <bool K16>
__global__ void probe(int trials, double* worst, int* bad) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int K = K16 ? 16 : 8;
  for (int it = 0; it < trials; ++it) {
    const unsigned base = ((blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * trials + it) * 4096u;
    __shared__ __half A[8][16][16], B[8][16][8];
    __shared__ float Cc[8][16][8];
    const int w = threadIdx.x / 32;
    for (int i = lane; i < 16 * K; i += 32) A[w][i / K][i % K] = rh(base + i);
    for (int i = lane; i < 8 * K; i += 32) B[w][i / 8][i % 8] = rh(base + 1000 + i);
    __syncwarp();
    const int mode = it % 3;  // 0: C = 0, 1: C cancels the product, 2: C random
    for (int i = lane; i < 128; i += 32) {
      const int r = i / 8, c = i % 8;
      double s = 0;
      for (int k = 0; k < K; ++k) s += (double)__half2float(A[w][r][k]) * (double)__half2float(B[w][k][c]);
      float cv = 0.f;
      if (mode == 1) cv = (float)(-s * (1.0 + 1e-3 * (urand(base + 3000 + i) - 0.5)));
      if (mode == 2) cv = ldexpf(urand(base + 3000 + i) - 0.5f, (int)(urand(base + 4000 + i) * 16) - 4);
      Cc[w][r][c] = cv;
    }
    __syncwarp();
    unsigned a0 = pk(A[w][g][2 * t], A[w][g][2 * t + 1]), a1 = pk(A[w][g + 8][2 * t], A[w][g + 8][2 * t + 1]);
    unsigned a2 = K16 ? pk(A[w][g][2 * t + 8], A[w][g][2 * t + 9]) : 0u, a3 = K16 ? pk(A[w][g + 8][2 * t + 8], A[w][g + 8][2 * t + 9]) : 0u;
    unsigned b0 = pk(B[w][2 * t][g], B[w][2 * t + 1][g]), b1 = K16 ? pk(B[w][2 * t + 8][g], B[w][2 * t + 9][g]) : 0u;
    float c0 = Cc[w][g][2 * t], c1 = Cc[w][g][2 * t + 1], c2 = Cc[w][g + 8][2 * t], c3 = Cc[w][g + 8][2 * t + 1];
    float d[4];
    if (K16)
      asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};\n"
          : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]) : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
    else
      asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%9,%10};\n"
          : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]) : "r"(a0), "r"(a1), "r"(b0), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
    for (int q = 0; q < 4; ++q) {
      const int r = g + (q >= 2 ? 8 : 0), c = 2 * t + (q & 1);
      double s = Cc[w][r][c], sa = fabs((double)Cc[w][r][c]);
      for (int k = 0; k < K; ++k) {
        const double p = (double)__half2float(A[w][r][k]) * (double)__half2float(B[w][k][c]);
        s += p; sa += fabs(p);
      }
      const double err = fabs((double)d[q] - s) / (sa > 0 ? sa : 1.0) * 16777216.0;
      if (err > 64.0) atomicAdd(bad, 1);
      // max via CAS on double bits (positive values order as integers)
      unsigned long long* wp = (unsigned long long*)worst + mode;
      unsigned long long v = __double_as_longlong(err), o = *wp;
      while (v > o) { unsigned long long p2 = atomicCAS(wp, o, v); if (p2 == o) break; o = p2; }
    }
    __syncwarp();
  }
}
int main() {
  double* w; int* bad;
  cudaMalloc(&w, 3 * sizeof(double)); cudaMalloc(&bad, sizeof(int));
  for (int k16 = 1; k16 >= 0; --k16) {
    cudaMemset(w, 0, 3 * sizeof(double)); cudaMemset(bad, 0, sizeof(int));
    if (k16) probe<true><<<304, 256>>>(200, w, bad); else probe<false><<<304, 256>>>(200, w, bad);
    cudaError_t e = cudaDeviceSynchronize();
    double hw[3]; int hb;
    cudaMemcpy(hw, w, sizeof hw, cudaMemcpyDeviceToHost); cudaMemcpy(&hb, bad, sizeof hb, cudaMemcpyDeviceToHost);
    printf("%s status=%d worst_c0=%.4f worst_cancel=%.4f worst_random=%.4f off=%d\n",
           k16 ? "m16n8k16" : "m16n8k8", (int)e, hw[0], hw[1], hw[2], hb);
  }
  return 0;
}
