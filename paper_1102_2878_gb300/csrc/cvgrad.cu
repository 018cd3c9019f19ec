// cvgrad.cu -- gradient of the leave-one-out likelihood score CV_LK with
// respect to log h and to every point, from exact sums.
//
// With K_ij = exp(-|x_i - x_j|^2 / 2h^2), S_i = sum_{j != i} K_ij and
// CV_LK = (1/N) sum_i log(S_i / ((N-1) V_{D,h})) (the introduction's
// likelihood cross-validation score), differentiating the definition gives
//   dCV/dlog h = (1/N) sum_i A_i / (h^2 S_i) - D,   A_i = sum_{j != i} K_ij |x_i - x_j|^2,
//   dCV/dx_k   = -(P_k / S_k + Y_k) / (N h^2),
//   P_k = sum_{j != k} K_kj (x_k - x_j),  Y_k = sum_{j != k} K_kj (x_k - x_j) / S_j.
// Every sum is over differences, so nothing cancels.  Two tiled passes over
// all pairs (the second needs every S_j), one thread per point, the other
// points staged in shared memory 256 at a time; kernel values in float32
// (ex2), each tile's partial sums added into float64 accumulators.
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kGT = 256;  // threads (points) per block and points per tile

// Pass 1: S_i, P_i (d values) and A_i of every point i; d <= DM.
template <int DM>
__global__ void __launch_bounds__(kGT) k_cvg_pass1(const float* __restrict__ X, int n, int d, float c2,
                                                   double* __restrict__ S, double* __restrict__ P,
                                                   double* __restrict__ A) {
  __shared__ float sX[kGT * DM];
  const int i = blockIdx.x * kGT + threadIdx.x;
  const bool have = i < n;
  float xi[DM];
#pragma unroll
  for (int k = 0; k < DM; ++k) xi[k] = (have && k < d) ? X[(size_t)i * d + k] : 0.f;
  double aS = 0.0, aA = 0.0, aP[DM];
#pragma unroll
  for (int k = 0; k < DM; ++k) aP[k] = 0.0;
  for (int t0 = 0; t0 < n; t0 += kGT) {
    const int tn = min(kGT, n - t0);
    for (int e = threadIdx.x; e < tn * d; e += kGT) sX[e] = X[(size_t)t0 * d + e];
    __syncthreads();
    float s = 0.f, a = 0.f, p[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) p[k] = 0.f;
    for (int j = 0; j < tn; ++j) {
      float df[DM], d2 = 0.f;
#pragma unroll
      for (int k = 0; k < DM; ++k) {
        df[k] = k < d ? xi[k] - sX[j * d + k] : 0.f;
        d2 = fmaf(df[k], df[k], d2);
      }
      const float K = (t0 + j == i) ? 0.f : ex2_approx(c2 * d2);
      s += K;
      a = fmaf(K, d2, a);
#pragma unroll
      for (int k = 0; k < DM; ++k) p[k] = fmaf(K, df[k], p[k]);
    }
    aS += s;
    aA += a;
#pragma unroll
    for (int k = 0; k < DM; ++k) aP[k] += p[k];
    __syncthreads();
  }
  if (have) {
    S[i] = aS;
    A[i] = aA;
#pragma unroll
    for (int k = 0; k < DM; ++k)
      if (k < d) P[(size_t)i * d + k] = aP[k];
  }
}

// Pass 2: Y_i = sum_{j != i} K_ij (x_i - x_j) / S_j; d <= DM.
template <int DM>
__global__ void __launch_bounds__(kGT) k_cvg_pass2(const float* __restrict__ X, int n, int d, float c2,
                                                   const double* __restrict__ S, double* __restrict__ Y) {
  __shared__ float sX[kGT * DM];
  __shared__ float sW[kGT];
  const int i = blockIdx.x * kGT + threadIdx.x;
  const bool have = i < n;
  float xi[DM];
#pragma unroll
  for (int k = 0; k < DM; ++k) xi[k] = (have && k < d) ? X[(size_t)i * d + k] : 0.f;
  double aY[DM];
#pragma unroll
  for (int k = 0; k < DM; ++k) aY[k] = 0.0;
  for (int t0 = 0; t0 < n; t0 += kGT) {
    const int tn = min(kGT, n - t0);
    for (int e = threadIdx.x; e < tn * d; e += kGT) sX[e] = X[(size_t)t0 * d + e];
    if (threadIdx.x < tn) sW[threadIdx.x] = (float)(1.0 / S[t0 + threadIdx.x]);
    __syncthreads();
    float y[DM];
#pragma unroll
    for (int k = 0; k < DM; ++k) y[k] = 0.f;
    for (int j = 0; j < tn; ++j) {
      float df[DM], d2 = 0.f;
#pragma unroll
      for (int k = 0; k < DM; ++k) {
        df[k] = k < d ? xi[k] - sX[j * d + k] : 0.f;
        d2 = fmaf(df[k], df[k], d2);
      }
      const float Kw = (t0 + j == i) ? 0.f : ex2_approx(c2 * d2) * sW[j];
#pragma unroll
      for (int k = 0; k < DM; ++k) y[k] = fmaf(Kw, df[k], y[k]);
    }
#pragma unroll
    for (int k = 0; k < DM; ++k) aY[k] += y[k];
    __syncthreads();
  }
  if (have) {
#pragma unroll
    for (int k = 0; k < DM; ++k)
      if (k < d) Y[(size_t)i * d + k] = aY[k];
  }
}

// Point gradients and per-block partial sums of log S_i and A_i / (h^2 S_i).
__global__ void __launch_bounds__(kGT) k_cvg_points(int n, int d, double h2, const double* __restrict__ S,
                                                    const double* __restrict__ A, const double* __restrict__ P,
                                                    const double* __restrict__ Y, double* __restrict__ dx,
                                                    double* __restrict__ part) {
  __shared__ double sL[kGT], sT[kGT];
  const int i = blockIdx.x * kGT + threadIdx.x;
  double l = 0.0, t = 0.0;
  if (i < n) {
    const double s = S[i];
    l = log(s);
    t = A[i] / (h2 * s);
    if (dx) {
      const double f = -1.0 / ((double)n * h2);
      for (int k = 0; k < d; ++k) dx[(size_t)i * d + k] = f * (P[(size_t)i * d + k] / s + Y[(size_t)i * d + k]);
    }
  }
  sL[threadIdx.x] = l;
  sT[threadIdx.x] = t;
  __syncthreads();
  for (int o = kGT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sL[threadIdx.x] += sL[threadIdx.x + o];
      sT[threadIdx.x] += sT[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sL[0];
    part[2 * blockIdx.x + 1] = sT[0];
  }
}

// Deterministic sum of the block partials: out = {sum log S, sum A/(h^2 S)}.
__global__ void k_cvg_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sL[kGT], sT[kGT];
  double l = 0.0, t = 0.0;
  for (int b = threadIdx.x; b < nb; b += kGT) {
    l += part[2 * b];
    t += part[2 * b + 1];
  }
  sL[threadIdx.x] = l;
  sT[threadIdx.x] = t;
  __syncthreads();
  for (int o = kGT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sL[threadIdx.x] += sL[threadIdx.x + o];
      sT[threadIdx.x] += sT[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sL[0];
    out[1] = sT[0];
  }
}

template <int DM>
void launch_passes(const float* X, int n, int d, float c2, double* S, double* P, double* A, double* Y, int nb,
                   cudaStream_t s) {
  k_cvg_pass1<DM><<<nb, kGT, 0, s>>>(X, n, d, c2, S, P, A);
  k_cvg_pass2<DM><<<nb, kGT, 0, s>>>(X, n, d, c2, S, Y);
}

}  // namespace

cudaError_t launch_cv_grad(const float* X, int n, int d, double h, double* S, double* P, double* A, double* Y,
                           double* part, double* out, double* dx, cudaStream_t s, long long* launches) {
  const int nb = (n + kGT - 1) / kGT;
  const float c2 = (float)(-kLog2e / (2.0 * h * h));
  switch (d) {
    case 1: launch_passes<1>(X, n, d, c2, S, P, A, Y, nb, s); break;
    case 2: launch_passes<2>(X, n, d, c2, S, P, A, Y, nb, s); break;
    case 3: launch_passes<3>(X, n, d, c2, S, P, A, Y, nb, s); break;
    case 4: launch_passes<4>(X, n, d, c2, S, P, A, Y, nb, s); break;
    case 5: launch_passes<5>(X, n, d, c2, S, P, A, Y, nb, s); break;
    default:
      if (d <= 8) launch_passes<8>(X, n, d, c2, S, P, A, Y, nb, s);
      else if (d <= 16) launch_passes<16>(X, n, d, c2, S, P, A, Y, nb, s);
      else launch_passes<32>(X, n, d, c2, S, P, A, Y, nb, s);
  }
  k_cvg_points<<<nb, kGT, 0, s>>>(n, d, h * h, S, A, P, Y, dx, part);
  k_cvg_final<<<1, kGT, 0, s>>>(part, nb, out);
  *launches += 4;
  return cudaGetLastError();
}

}  // namespace dfgt
