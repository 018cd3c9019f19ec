// bruteforce.cu -- exact Gaussian sums by the all-pairs loop of Algorithm 1
// (NaiveKDE without its normalisation), for several bandwidths at once.
//
// One thread owns one query; the block streams reference tiles through
// shared memory, stored negated as structure-of-arrays so one 64-bit load
// gives one coordinate of two consecutive references.  The squared
// distances of the two pairs (direct differences) are formed with packed
// f32x2 add / fma and reused for every bandwidth of the chunk:
// exp(-d2/2h^2) = 2^(d2 * c_h), c_h = -log2(e)/(2h^2), on the SFU.  With
// n_h bandwidths a pair of references costs 2D + 2 n_h packed FP32 ops and
// 2 n_h ex2, so the loop is bound by the ex2 rate.  Each run of 32
// references is summed in float32 and the runs are added with Kahan
// compensation.
//
// A query set too small to fill the GPU splits the references into slices
// over blockIdx.y; each slice writes float64 partial sums to scratch
// memory and a second kernel adds the slices in a fixed order.
#include <algorithm>

#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kBfThreads = 128;
constexpr int kBfTile = 128;           // references per shared-memory tile (even)
constexpr float kFarNeg = -1.0e18f;    // padding reference: contributes 0
constexpr int kSplitTargetBlocks = 152 * 8;  // blocks that keep every SM busy
constexpr int kMaxSlices = 256;

// Reference slicing of one launch: `slices` slices of `len` references;
// slice s writes its partial sums at G + s * stride.
struct Split {
  int slices;
  int len;
  size_t stride;
};

template <int NHB>
struct HChunk {
  float c[NHB];
};

template <int D, int NHB>
__global__ void __launch_bounds__(kBfThreads) k_bruteforce(const float* __restrict__ q, int nq,
                                                           const float* __restrict__ r, int nr,
                                                           HChunk<NHB> hc, double* __restrict__ G,
                                                           int ldg, int slice_len,
                                                           size_t slice_stride) {
  __shared__ __align__(16) float sr[D][kBfTile];
  const int qi = blockIdx.x * kBfThreads + threadIdx.x;
  // reference slice of this block (blockIdx.y); the whole set when unsplit
  r += (size_t)blockIdx.y * slice_len * D;
  nr = min(slice_len, nr - (int)blockIdx.y * slice_len);
  G += blockIdx.y * slice_stride;
  float2 qq[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float v = qi < nq ? q[(size_t)qi * D + k] : 0.f;
    qq[k] = make_float2(v, v);
  }
  float2 cp[NHB];
  float S[NHB], C[NHB];
#pragma unroll
  for (int hh = 0; hh < NHB; ++hh) {
    cp[hh] = make_float2(hc.c[hh], hc.c[hh]);
    S[hh] = C[hh] = 0.f;
  }
  for (int t0 = 0; t0 < nr; t0 += kBfTile) {
    const int tn = min(kBfTile, nr - t0);
    const int tn2 = (tn + 1) & ~1;
    __syncthreads();
    for (int e = threadIdx.x; e < tn2 * D; e += kBfThreads) {
      const int j = e / D, k = e % D;
      sr[k][j] = j < tn ? -r[(size_t)(t0 + j) * D + k] : kFarNeg;
    }
    __syncthreads();
    for (int j0 = 0; j0 < tn2; j0 += 32) {
      const int je = min(j0 + 32, tn2);
      float2 part[NHB];
#pragma unroll
      for (int hh = 0; hh < NHB; ++hh) part[hh] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int j = j0; j < je; j += 2) {
        float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float2 rr = *reinterpret_cast<const float2*>(&sr[k][j]);
          const float2 dd = __fadd2_rn(qq[k], rr);
          d2 = __ffma2_rn(dd, dd, d2);
        }
#pragma unroll
        for (int hh = 0; hh < NHB; ++hh) {
          const float2 a = __fmul2_rn(d2, cp[hh]);
          part[hh] = __fadd2_rn(part[hh], make_float2(ex2_approx(a.x), ex2_approx(a.y)));
        }
      }
#pragma unroll
      for (int hh = 0; hh < NHB; ++hh) {
        const float y = (part[hh].x + part[hh].y) - C[hh];
        const float t = S[hh] + y;
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

// Any dimension up to 32, scalar math (dimensions above 5 are not the
// exp-bound case: the 2D distance flops dominate there).
template <int NHB>
__global__ void __launch_bounds__(kBfThreads) k_bruteforce_g(const float* __restrict__ q, int nq,
                                                             const float* __restrict__ r, int nr,
                                                             int d, HChunk<NHB> hc,
                                                             double* __restrict__ G, int ldg,
                                                             int slice_len, size_t slice_stride) {
  __shared__ float sr[kBfTile * kMaxD];
  const int qi = blockIdx.x * kBfThreads + threadIdx.x;
  r += (size_t)blockIdx.y * slice_len * d;
  nr = min(slice_len, nr - (int)blockIdx.y * slice_len);
  G += blockIdx.y * slice_stride;
  float qv[kMaxD];
#pragma unroll
  for (int k = 0; k < kMaxD; ++k) qv[k] = (k < d && qi < nq) ? q[(size_t)qi * d + k] : 0.f;
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
      for (int j = j0; j < je; ++j) {
        float d2 = 0.f;
#pragma unroll
        for (int k = 0; k < kMaxD; ++k) {
          if (k < d) {
            const float t = qv[k] - sr[j * d + k];
            d2 = fmaf(t, t, d2);
          }
        }
#pragma unroll
        for (int hh = 0; hh < NHB; ++hh) part[hh] += ex2_approx(d2 * hc.c[hh]);
      }
#pragma unroll
      for (int hh = 0; hh < NHB; ++hh) {
        const float y = part[hh] - C[hh];
        const float t = S[hh] + y;
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
                         double* G, int ldg, const Split& sp, cudaStream_t s) {
  HChunk<NHB> hc;
  for (int i = 0; i < NHB; ++i) hc.c[i] = (float)(-kLog2e / (2.0 * h[i] * h[i]));
  const dim3 grid((nq + kBfThreads - 1) / kBfThreads, sp.slices);
  if constexpr (D > 0)
    k_bruteforce<D, NHB><<<grid, kBfThreads, 0, s>>>(q, nq, r, nr, hc, G, ldg, sp.len, sp.stride);
  else
    k_bruteforce_g<NHB><<<grid, kBfThreads, 0, s>>>(q, nq, r, nr, d, hc, G, ldg, sp.len, sp.stride);
  return cudaGetLastError();
}

// Bandwidths are processed in chunks whose sizes have a compiled variant;
// the largest variant that fits the remainder is taken.  Out is either the
// result [nh][nq] or, when split, the slice partials [slices][nh][nq].
template <int D>
cudaError_t launch_d(const float* q, int nq, const float* r, int nr, int d, const double* h,
                     int nh, double* out, const Split& sp, cudaStream_t s, long long* launches) {
  int done = 0;
  while (done < nh) {
    const int rem = nh - done;
    const double* hp = h + done;
    double* Gp = out + (size_t)done * nq;
    cudaError_t e;
    int take;
    if (rem >= 16) { take = 16; e = launch_chunk<D, 16>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    else if (rem >= 12) { take = 12; e = launch_chunk<D, 12>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    else if (rem >= 10) { take = 10; e = launch_chunk<D, 10>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    else if (rem >= 8) { take = 8; e = launch_chunk<D, 8>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    else if (rem >= 6) { take = 6; e = launch_chunk<D, 6>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    else if (rem >= 4) { take = 4; e = launch_chunk<D, 4>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    else if (rem >= 2) { take = 2; e = launch_chunk<D, 2>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    else { take = 1; e = launch_chunk<D, 1>(q, nq, r, nr, d, hp, Gp, nq, sp, s); }
    ++*launches;
    if (e != cudaSuccess) return e;
    done += take;
  }
  return cudaSuccess;
}

// Sum the slice partials [slices][total] in slice order into G[total].
__global__ void k_reduce_slices(const double* __restrict__ part, int slices, long total,
                                double* __restrict__ G) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  double acc = 0.0;
  for (int sl = 0; sl < slices; ++sl) acc += part[(size_t)sl * total + i];
  G[i] = acc;
}

cudaError_t dispatch(const float* q, int nq, const float* r, int nr, int d, const double* h, int nh,
                     double* out, const Split& sp, cudaStream_t s, long long* launches) {
  switch (d) {
    case 1: return launch_d<1>(q, nq, r, nr, d, h, nh, out, sp, s, launches);
    case 2: return launch_d<2>(q, nq, r, nr, d, h, nh, out, sp, s, launches);
    case 3: return launch_d<3>(q, nq, r, nr, d, h, nh, out, sp, s, launches);
    case 4: return launch_d<4>(q, nq, r, nr, d, h, nh, out, sp, s, launches);
    case 5: return launch_d<5>(q, nq, r, nr, d, h, nh, out, sp, s, launches);
    default: return launch_d<0>(q, nq, r, nr, d, h, nh, out, sp, s, launches);
  }
}

}  // namespace

int bruteforce_slices(int nq, int nr) {
  const int qblocks = (nq + kBfThreads - 1) / kBfThreads;
  if (qblocks >= 2 * kSplitTargetBlocks / 8) return 1;  // the queries fill the GPU
  int sl = (kSplitTargetBlocks + qblocks - 1) / qblocks;
  const int max_by_r = (nr + kBfTile - 1) / kBfTile;  // at least one tile per slice
  sl = std::min(sl, std::min(max_by_r, kMaxSlices));
  return std::max(sl, 1);
}

cudaError_t launch_bruteforce_split(const float* q, int nq, const float* r, int nr, int d,
                                    const double* h_host, int nh, double* G, int slices,
                                    double* partials, cudaStream_t s, long long* launches) {
  Split sp{1, nr, 0};
  if (slices <= 1) return dispatch(q, nq, r, nr, d, h_host, nh, G, sp, s, launches);
  // slice lengths are whole tiles, so every slice but the last is full
  const int tiles = (nr + kBfTile - 1) / kBfTile;
  const int per = (tiles + slices - 1) / slices;
  sp.len = per * kBfTile;
  sp.slices = (nr + sp.len - 1) / sp.len;
  sp.stride = (size_t)nh * nq;
  cudaError_t e = dispatch(q, nq, r, nr, d, h_host, nh, partials, sp, s, launches);
  if (e != cudaSuccess) return e;
  const long total = (long)nh * nq;
  k_reduce_slices<<<(int)((total + 255) / 256), 256, 0, s>>>(partials, sp.slices, total, G);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_bruteforce(const float* q, int nq, const float* r, int nr, int d,
                              const double* h_host, int nh, double* G, DevBuf& scratch,
                              cudaStream_t s, long long* launches) {
  const int slices = bruteforce_slices(nq, nr);
  double* partials = nullptr;
  if (slices > 1) {
    cudaError_t e = scratch.ensure((size_t)slices * nh * nq * sizeof(double));
    if (e != cudaSuccess) return e;
    partials = scratch.as<double>();
  }
  return launch_bruteforce_split(q, nq, r, nr, d, h_host, nh, G, slices, partials, s, launches);
}

}  // namespace dfgt
