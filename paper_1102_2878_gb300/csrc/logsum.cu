// logsum.cu -- log G for queries whose Gaussian sum (Eq. 5) lies below the
// range the dual-tree pass resolves.
//
// The relative guarantee of Definition 1.2 is per query, but a query far
// from every reference (bichromatic sets, small h, large D) has a sum far
// below the float32 range of the exact leaf sums, often below the float64
// range too.  Such a sum is carried in log form with a per-query shift:
// with x_j = |q - r_j|^2 / 2h^2 and m = min_j x_j,
//     log G(q) = -m + log sum_j exp(-(x_j - m)),
// where every shifted term is <= 1 and the nearest one is exactly 1.
//
// After the dual-tree pass, every (bandwidth, query) whose estimate is
// below kLogFlag is listed (k_log_flag), bandwidths in chunks of 16 with a
// bit mask per query.  One warp per listed (query, chunk) walks the
// reference tree depth first, nearer child first, from the root
// (k_log_sum):
//   * a node whose squared box distance d^l satisfies
//     d^l >= m2 + 2 h_max^2 T (m2 the smallest squared distance found so
//     far, h_max the largest listed bandwidth) is skipped: each of its
//     points adds at most exp(-T) G, so with T = log(|R| / eps_skip) + 1 the
//     skipped part of the sum is below eps_skip G (the finite-difference
//     prune of the traversal with value 0, in shifted form);
//   * at a leaf the lanes take 32 points at a time; each squared distance
//     is a double-float (hi + lo) from exact differences (Knuth's TwoSum)
//     and exact squares (FMA), so x_j - m keeps its absolute accuracy
//     even when x_j is in the thousands; the warp minimum updates m2 (the
//     running sums are rescaled by exp(-(m_old - m_new)/2h^2)), and every
//     lane adds exp2(-(x_j - m) log2 e) per listed bandwidth.
// The result is written as log G and as G = exp(log G) in float64 (which
// underflows to 0 where G does).
#include <cmath>

#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kLogWarps = 8;     // warps per block
constexpr int kLogChunk = 16;    // bandwidths per listed item
constexpr int kLogStack = 192;   // depth-first stack per warp (tree depth <= 128 levels)

struct LogItem {
  int q;      // query position in the query tree (permuted order)
  int chunk;  // bandwidths [16 chunk, 16 chunk + 16)
  int mask;   // which of them are listed
  int pad;
};

// Flag every (bandwidth, query) whose estimate is below `flag`; one item per
// query and chunk of 16 bandwidths with a nonempty mask.
__global__ void k_log_flag(const double* __restrict__ G, int nq, int nh, const int* __restrict__ perm,
                           double flag, LogItem* __restrict__ items, int* __restrict__ n_items,
                           unsigned long long* __restrict__ n_flagged) {
  const int nchunks = (nh + kLogChunk - 1) / kLogChunk;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)nq * nchunks;
  int mask = 0;
  int qi = 0, c = 0;
  if (t < total) {
    qi = (int)(t / nchunks);
    c = (int)(t % nchunks);
    const int orig = perm[qi];
    for (int k = 0; k < kLogChunk; ++k) {
      const int h = c * kLogChunk + k;
      if (h < nh && !(G[(size_t)h * nq + orig] >= flag)) mask |= 1 << k;
    }
  }
  const unsigned FULL = 0xffffffffu;
  const unsigned has = __ballot_sync(FULL, mask != 0);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && has) base = atomicAdd(n_items, __popc(has));
  base = __shfl_sync(FULL, base, 0);
  if (mask) {
    items[base + __popc(has & ((1u << lane) - 1u))] = LogItem{qi, c, mask, 0};
    atomicAdd(n_flagged, (unsigned long long)__popc(mask));
  }
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Squared distance of two points as a double-float hi + lo, accurate to a
// few units of 2^-44 relative.
template <int DM>
__device__ __forceinline__ double dist2_df(const float* q, const float* r) {
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int k = 0; k < DM; ++k) {
    float s, e;
    two_sum(q[k], -r[k], s, e);  // s + e = q - r exactly
    const float p = s * s;
    const float pe = fmaf(s, s, -p);  // s^2 = p + pe exactly
    float t, te;
    two_sum(hi, p, t, te);
    hi = t;
    lo += te + pe;
    lo = fmaf(2.f * s, e, lo);  // (s + e)^2 - s^2 up to e^2
  }
  return (double)hi + (double)lo;
}

template <int DM>
__device__ __forceinline__ void load_row(const float* __restrict__ p, int dp, float* v) {
  if constexpr (DM >= 4) {
#pragma unroll
    for (int k4 = 0; k4 < DM / 4; ++k4) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4 * k4 < dp) a = __ldg(reinterpret_cast<const float4*>(p) + k4);
      v[4 * k4] = a.x;
      v[4 * k4 + 1] = a.y;
      v[4 * k4 + 2] = a.z;
      v[4 * k4 + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < DM; ++k) v[k] = k < dp ? __ldg(p + k) : 0.f;
  }
}

// Lower bound on the squared distance from q to node `node`'s box: lane k
// holds dimension k; the float sum is scaled down by 2^-16 for its rounding.
__device__ __forceinline__ float box_dl2(const TreeView& R, int node, float qk, int lane) {
  float g2 = 0.f;
  if (lane < R.d) {
    const float lo = R.lo[(size_t)node * R.d + lane], hi = R.hi[(size_t)node * R.d + lane];
    const float gap = fmaxf(0.f, fmaxf(__fsub_rd(lo, qk), __fsub_rd(qk, hi)));
    g2 = __fmul_rd(gap, gap);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g2 += __shfl_xor_sync(0xffffffffu, g2, o);
  return g2 * (1.f - 1.0f / 65536.f);
}

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

struct LogArgs {
  TreeView Q, R;
  const LogItem* items;
  const int* n_items;
  const double* h;        // [nh]
  double* G;              // [nh][nq] caller order
  double* logG;           // [nh][nq] caller order
  int* status;
  int nh;
  float T;                // skip margin in units of 2 h^2 (natural log)
};

template <int DM>
__global__ void __launch_bounds__(kLogWarps * 32) k_log_sum(LogArgs A) {
  __shared__ int sStack[kLogWarps][kLogStack];
  const unsigned FULL = 0xffffffffu;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = *A.n_items;
  const TreeView& Q = A.Q;
  const TreeView& R = A.R;
  int* stack = sStack[wib];
  for (int it = blockIdx.x * kLogWarps + wib; it < n_items; it += gridDim.x * kLogWarps) {
    const LogItem item = A.items[it];
    float q[DM];
    load_row<DM>(Q.pts + (size_t)item.q * Q.dp, Q.dp, q);
    const float qk = lane < Q.d ? Q.pts[(size_t)item.q * Q.dp + lane] : 0.f;
    // per-bandwidth exp2 scales log2(e)/2h^2 and the skip radius of the largest listed h
    float c2[kLogChunk];
    float hmax = 0.f;
#pragma unroll
    for (int k = 0; k < kLogChunk; ++k) {
      const int hi = item.chunk * kLogChunk + k;
      const bool on = (item.mask >> k) & 1;
      const double h = on ? A.h[hi] : 1.0;
      c2[k] = on ? (float)(kLog2e / (2.0 * h * h)) : 0.f;
      if (on) hmax = fmaxf(hmax, (float)h);
    }
    const float rad2 = 2.f * hmax * hmax * A.T * 1.0001f;
    double m2 = INFINITY;  // smallest squared distance so far
    double S[kLogChunk];
#pragma unroll
    for (int k = 0; k < kLogChunk; ++k) S[k] = 0.0;
    int sp = 0;
    if (lane == 0) stack[0] = 0;
    sp = 1;
    __syncwarp();
    while (sp > 0) {
      const int node = stack[--sp];
      __syncwarp();
      const float dl2 = box_dl2(R, node, qk, lane);
      if ((double)dl2 > m2 + (double)rad2) continue;
      const int left = R.left[node];
      if (left >= 0) {
        const float d0 = box_dl2(R, left, qk, lane), d1 = box_dl2(R, left + 1, qk, lane);
        const bool k0 = (double)d0 <= m2 + (double)rad2, k1 = (double)d1 <= m2 + (double)rad2;
        // push the farther child first, so the nearer one is visited next
        const int nearc = d0 <= d1 ? left : left + 1, farc = d0 <= d1 ? left + 1 : left;
        const bool knear = d0 <= d1 ? k0 : k1, kfar = d0 <= d1 ? k1 : k0;
        if (sp + 2 > kLogStack) {  // cannot happen for trees of <= 128 levels
          if (lane == 0) atomicOr(A.status, kStOverflow);
          break;
        }
        if (lane == 0) {
          if (kfar) stack[sp] = farc;
          if (knear) stack[sp + (kfar ? 1 : 0)] = nearc;
        }
        sp += (kfar ? 1 : 0) + (knear ? 1 : 0);
        __syncwarp();
        continue;
      }
      // a leaf: 32 points at a time
      const int rb = R.beg[node], rn = R.cnt[node];
      float part[kLogChunk];
#pragma unroll
      for (int k = 0; k < kLogChunk; ++k) part[k] = 0.f;
      for (int j0 = 0; j0 < rn; j0 += 32) {
        const int j = j0 + lane;
        double d2 = INFINITY;
        if (j < rn) {
          float r[DM];
          load_row<DM>(R.pts + (size_t)(rb + j) * R.dp, R.dp, r);
          d2 = dist2_df<DM>(q, r);
        }
        const double mn = warp_min_d(d2);
        if (mn < m2) {
          // a nearer point: rescale what was summed relative to the old shift
          const float drop = m2 == INFINITY ? INFINITY : (float)(m2 - mn);
#pragma unroll
          for (int k = 0; k < kLogChunk; ++k) {
            const float f = drop == INFINITY ? 0.f : ex2_approx(-drop * c2[k]);
            S[k] *= (double)f;
            part[k] *= f;
          }
          m2 = mn;
        }
        if (j < rn) {
          const float t = (float)(d2 - m2);  // >= 0, accurate to its own rounding
#pragma unroll
          for (int k = 0; k < kLogChunk; ++k)
            if ((item.mask >> k) & 1) part[k] += ex2_approx(-t * c2[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < kLogChunk; ++k) S[k] += (double)part[k];
    }
    // reduce the lanes' sums and write log G = -m2/2h^2 + log S and G
#pragma unroll
    for (int k = 0; k < kLogChunk; ++k) {
      double v = S[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
      S[k] = v;
    }
    const int orig = Q.perm[item.q];
    const int nq = Q.n;
#pragma unroll
    for (int k = 0; k < kLogChunk; ++k) {
      if (lane == k && ((item.mask >> k) & 1)) {
        const int hi = item.chunk * kLogChunk + k;
        const double h = A.h[hi];
        const double lg = -m2 / (2.0 * h * h) + log(S[k]);
        A.logG[(size_t)hi * nq + orig] = lg;
        A.G[(size_t)hi * nq + orig] = exp(lg);
      }
    }
    __syncwarp();
  }
}

// log G of every (bandwidth, query) not listed: the log of the estimate.
__global__ void k_log_plain(const double* __restrict__ G, long total, double* __restrict__ logG, double flag) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) {
    const double g = G[i];
    if (g >= flag) logG[i] = log(g);
  }
}

}  // namespace

cudaError_t launch_log_pass(const TreeView& Q, const TreeView& R, const double* h_dev, int nh, double eps,
                            double flag, double* G, double* logG, DevBuf& items_buf, int* counters,
                            unsigned long long* n_flagged, int* status, cudaStream_t s, long long* launches,
                            int* n_items_host) {
  const int nq = Q.n;
  const int nchunks = (nh + kLogChunk - 1) / kLogChunk;
  const long total_items = (long)nq * nchunks;
  cudaError_t e = items_buf.ensure((size_t)total_items * sizeof(LogItem));
  if (e != cudaSuccess) return e;
  LogItem* items = items_buf.as<LogItem>();
  const long total = (long)nh * nq;
  k_log_plain<<<(int)((total + 255) / 256), 256, 0, s>>>(G, total, logG, flag);
  if ((e = cudaMemsetAsync(counters, 0, sizeof(int), s)) != cudaSuccess) return e;
  k_log_flag<<<(int)((total_items + 255) / 256), 256, 0, s>>>(G, nq, nh, Q.perm, flag, items, counters, n_flagged);
  *launches += 2;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(n_items_host, counters, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  const int n = *n_items_host;
  if (n == 0) return cudaSuccess;
  LogArgs A;
  A.Q = Q;
  A.R = R;
  A.items = items;
  A.n_items = counters;
  A.h = h_dev;
  A.G = G;
  A.logG = logG;
  A.status = status;
  A.nh = nh;
  // skipped points add at most |R| exp(-T) G <= (eps / 4) G
  A.T = (float)(std::log((double)R.n) - std::log(0.25 * eps) + 1.0);
  const int grid = (int)std::min<long>((n + kLogWarps - 1) / kLogWarps, 152L * 64);
  const int dp = std::max(Q.dp, R.dp);
  if (dp <= 2) k_log_sum<2><<<grid, kLogWarps * 32, 0, s>>>(A);
  else if (dp <= 4) k_log_sum<4><<<grid, kLogWarps * 32, 0, s>>>(A);
  else if (dp <= 8) k_log_sum<8><<<grid, kLogWarps * 32, 0, s>>>(A);
  else if (dp <= 16) k_log_sum<16><<<grid, kLogWarps * 32, 0, s>>>(A);
  else k_log_sum<32><<<grid, kLogWarps * 32, 0, s>>>(A);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace dfgt
