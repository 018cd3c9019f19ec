// bruteforce.cu -- exact Gaussian sums by the all-pairs loop of Algorithm 1
// (NaiveKDE without its normalisation), for several bandwidths at once.
//
// One thread owns one query; the block streams reference tiles through
// shared memory.  The squared distance of a pair is computed once (direct
// differences, float32) and reused for every bandwidth of the chunk:
// exp(-d2/2h^2) = 2^(d2 * c_h) with c_h = -log2(e)/(2h^2) on the SFU.
// Each run of 32 references is summed in float32 and the runs are added
// with Kahan compensation, so the result is accurate to a few float32 ulps.
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kBfThreads = 128;
constexpr int kBfTile = 128;

template <int NHB>
struct HChunk {
  float c[NHB];
};

template <int D, int NHB>
__global__ void __launch_bounds__(kBfThreads) k_bruteforce(const float* __restrict__ q, int nq,
                                                           const float* __restrict__ r, int nr,
                                                           int d_rt, HChunk<NHB> hc,
                                                           double* __restrict__ G, int ldg) {
  constexpr int DD = D > 0 ? D : kMaxD;
  const int d = D > 0 ? D : d_rt;
  __shared__ float sr[kBfTile * DD];
  const int qi = blockIdx.x * kBfThreads + threadIdx.x;
  float qv[DD];
#pragma unroll
  for (int k = 0; k < DD; ++k) qv[k] = (k < d && qi < nq) ? q[(size_t)qi * d + k] : 0.f;
  float S[NHB], C[NHB];
#pragma unroll
  for (int hh = 0; hh < NHB; ++hh) S[hh] = C[hh] = 0.f;

  for (int t0 = 0; t0 < nr; t0 += kBfTile) {
    const int tn = min(kBfTile, nr - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < tn * d; e += kBfThreads) sr[e] = r[(size_t)t0 * d + e];
    __syncthreads();
    for (int j0 = 0; j0 < tn; j0 += 32) {
      const int je = min(j0 + 32, tn);
      float part[NHB];
#pragma unroll
      for (int hh = 0; hh < NHB; ++hh) part[hh] = 0.f;
#pragma unroll 4
      for (int j = j0; j < je; ++j) {
        float d2 = 0.f;
#pragma unroll
        for (int k = 0; k < DD; ++k) {
          if (k < d) {
            float t = qv[k] - sr[j * d + k];
            d2 = fmaf(t, t, d2);
          }
        }
#pragma unroll
        for (int hh = 0; hh < NHB; ++hh) part[hh] += ex2_approx(d2 * hc.c[hh]);
      }
#pragma unroll
      for (int hh = 0; hh < NHB; ++hh) {
        float y = part[hh] - C[hh];
        float t = S[hh] + y;
        C[hh] = (t - S[hh]) - y;
        S[hh] = t;
      }
    }
  }
  if (qi < nq) {
#pragma unroll
    for (int hh = 0; hh < NHB; ++hh) G[(size_t)hh * ldg + qi] = (double)S[hh] - (double)C[hh];
  }
}

template <int D, int NHB>
cudaError_t launch_chunk(const float* q, int nq, const float* r, int nr, int d, const double* h,
                         double* G, int ldg, cudaStream_t s) {
  HChunk<NHB> hc;
  for (int i = 0; i < NHB; ++i) hc.c[i] = (float)(-kLog2e / (2.0 * h[i] * h[i]));
  const int grid = (nq + kBfThreads - 1) / kBfThreads;
  k_bruteforce<D, NHB><<<grid, kBfThreads, 0, s>>>(q, nq, r, nr, d, hc, G, ldg);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_d(const float* q, int nq, const float* r, int nr, int d, const double* h,
                     int nh, double* G, cudaStream_t s, long long* launches) {
  int done = 0;
  while (done < nh) {
    const int rem = nh - done;
    cudaError_t e;
    int take;
    if (rem >= 16) { take = 16; e = launch_chunk<D, 16>(q, nq, r, nr, d, h + done, G + (size_t)done * nq, nq, s); }
    else if (rem >= 8) { take = 8; e = launch_chunk<D, 8>(q, nq, r, nr, d, h + done, G + (size_t)done * nq, nq, s); }
    else if (rem >= 4) { take = 4; e = launch_chunk<D, 4>(q, nq, r, nr, d, h + done, G + (size_t)done * nq, nq, s); }
    else if (rem >= 2) { take = 2; e = launch_chunk<D, 2>(q, nq, r, nr, d, h + done, G + (size_t)done * nq, nq, s); }
    else { take = 1; e = launch_chunk<D, 1>(q, nq, r, nr, d, h + done, G + (size_t)done * nq, nq, s); }
    ++*launches;
    if (e != cudaSuccess) return e;
    done += take;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_bruteforce(const float* q, int nq, const float* r, int nr, int d,
                              const double* h_host, int nh, double* G, cudaStream_t s,
                              long long* launches) {
  switch (d) {
    case 1: return launch_d<1>(q, nq, r, nr, d, h_host, nh, G, s, launches);
    case 2: return launch_d<2>(q, nq, r, nr, d, h_host, nh, G, s, launches);
    case 3: return launch_d<3>(q, nq, r, nr, d, h_host, nh, G, s, launches);
    case 4: return launch_d<4>(q, nq, r, nr, d, h_host, nh, G, s, launches);
    case 5: return launch_d<5>(q, nq, r, nr, d, h_host, nh, G, s, launches);
    default: return launch_d<0>(q, nq, r, nr, d, h_host, nh, G, s, launches);
  }
}

}  // namespace dfgt
