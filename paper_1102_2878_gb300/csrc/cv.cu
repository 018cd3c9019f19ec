// cv.cu -- cross-validation scores of a bandwidth sweep from dual-tree sums
// over one point set (Q = R): the likelihood score CV_LK and the
// least-squares score CV_LS of the paper's introduction, with the density
// estimate of Eq. 1 (Gaussian kernel, V_{D,h} = (2 pi h^2)^{D/2}).
//
// The inputs are the leave-one-out sums S_i (dfgt_sum_loo, Q = R, each
// point's own term left out) over the bandwidths h and sqrt(2) h (the
// convolution kernel K_h * K_h of CV_LS is the Gaussian of deviation
// sqrt(2) h):
//   CV_LK(h) = (1/N) sum_i log(S_i / ((N-1) V_{D,h}))
//   CV_LS(h) = (1/N) sum_i (S*_i / ((N-1) V_{D,sqrt2 h}) - 2 S_i / ((N-1) V_{D,h})).
// The sums carry |S~ - S| <= eps S, so |log S~ - log S| <= -log(1 - eps)
// and |S~ - S| <= eps' S~ with eps' = eps / (1 - eps); the CV_LS error is
// linear in the sums.  Both bounds are accumulated beside the scores.  The
// reduction
// is float64 and runs in a fixed order (per-block partials, then one pass
// per bandwidth), so scores are reproducible.
#include <cmath>

#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kT = 256;
constexpr int kTerms = 4;  // sum log S~, sum of log bounds, sum of CV_LS terms, sum of their bounds

__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kT / 32; ++w) t += scratch[w];
  __syncthreads();
  return t;  // valid in thread 0
}

// G: [2 nh][n] leave-one-out sums, rows k < nh at h_k and rows nh + k at sqrt(2) h_k.
// norm: [2 nh] (n - 1) V for the same rows.  part: [nh][gridDim.x][kTerms].
__global__ void __launch_bounds__(kT) k_cv_partials(const double* __restrict__ G, int n, int nh,
                                                    const double* __restrict__ norm, double epsp,
                                                    double* __restrict__ part) {
  __shared__ double scratch[kT / 32];
  const int k = blockIdx.y;
  const double* g = G + (size_t)k * n;
  const double* gs = G + (size_t)(nh + k) * n;
  const double nv = norm[k], nvs = norm[nh + k];
  double t[kTerms] = {0.0, 0.0, 0.0, 0.0};
  const double eps = epsp / (1.0 + epsp);
  for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) {
    const double S = g[i], Ss = gs[i];
    t[0] += S > 0.0 ? log(S) : -INFINITY;
    t[1] += S > 0.0 ? -log1p(-eps) : INFINITY;
    t[2] += Ss / nvs - 2.0 * S / nv;
    t[3] += epsp * (Ss / nvs + 2.0 * S / nv);
  }
#pragma unroll
  for (int q = 0; q < kTerms; ++q) {
    const double v = block_sum(t[q], scratch);
    if (threadIdx.x == 0) part[((size_t)k * gridDim.x + blockIdx.x) * kTerms + q] = v;
  }
}

// out: [nh][4] = CV_LK, its bound, CV_LS, its bound.
__global__ void k_cv_final(const double* __restrict__ part, int nblk, int nh, int n,
                           const double* __restrict__ norm, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nh) return;
  double s[kTerms] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < nblk; ++b)
#pragma unroll
    for (int q = 0; q < kTerms; ++q) s[q] += part[((size_t)k * nblk + b) * kTerms + q];
  out[k * 4 + 0] = s[0] / n - log(norm[k]);
  out[k * 4 + 1] = s[1] / n;
  out[k * 4 + 2] = s[2] / n;
  out[k * 4 + 3] = s[3] / n;
}

}  // namespace

cudaError_t launch_cv_scores(const double* G, int n, int nh, const double* norm, double eps, double* part,
                             int nblk, double* out, cudaStream_t s, long long* launches) {
  const double epsp = eps / (1.0 - eps);
  k_cv_partials<<<dim3(nblk, nh), kT, 0, s>>>(G, n, nh, norm, epsp, part);
  k_cv_final<<<(nh + 63) / 64, 64, 0, s>>>(part, nblk, nh, n, norm, out);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace dfgt
