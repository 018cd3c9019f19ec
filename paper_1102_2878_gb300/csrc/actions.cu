// actions.cu -- the summaries and exact sums the traversal decided on
// (Summarize and DFGTBase of Section 3.6) and the post-processing pass
// (DFGTPost: local-to-local translation down the query tree, local
// expansion read-out, final sum).
//
// One warp handles one listed node pair.  Multi-index tables use the
// paper's linear layout (radix p_max, last dimension least significant)
// and are unrolled at compile time per dimension D = 1..5; D >= 6 has
// p_max = 1 and uses the order-0 kernels at the end of the file.  Sums of
// the exact and far-field parts go to a float64 per-query accumulator;
// local moments are float64 per (bandwidth, query node).
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kT = 256;
constexpr int kWarpsPerBlock = kT / 32;

template <int D, int PM>
__device__ __forceinline__ constexpr int digit_c(int idx, int k) {
  int v = idx;
  for (int j = D - 1; j > k; --j) v /= PM;
  return v % PM;
}

template <int D, int PM>
__device__ __forceinline__ int abs_c(int idx) {
  int s = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) s += digit_c<D, PM>(idx, k);
  return s;
}

template <int D, int PM>
__device__ __forceinline__ bool below_c(int idx, int p) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < D; ++k) ok = ok && (digit_c<D, PM>(idx, k) < p);
  return ok;
}

template <int D, int PM>
__device__ __forceinline__ double multifact_c(int idx) {
  double f = 1.0;
#pragma unroll
  for (int k = 0; k < D; ++k) f *= fact_d(digit_c<D, PM>(idx, k));
  return f;
}

// Hermite functions h_0..h_{NT-1}(t) (h_n = e^{-t^2} H_n(t)) by the
// recurrence h_{n+1} = 2t h_n - 2n h_{n-1} (ComputePartialDerivatives).
template <int NT>
__device__ __forceinline__ void hermite_f32(float t, float* H) {
  H[0] = ex2_approx(-t * t * (float)kLog2e);
  if (NT > 1) H[1] = 2.f * t * H[0];
#pragma unroll
  for (int n = 1; n + 1 < NT; ++n) H[n + 1] = 2.f * t * H[n] - 2.f * (float)n * H[n - 1];
}

template <int NT>
__device__ __forceinline__ void hermite_f64(double t, double* H) {
  H[0] = exp(-t * t);
  if (NT > 1) H[1] = 2.0 * t * H[0];
#pragma unroll
  for (int n = 1; n + 1 < NT; ++n) H[n + 1] = 2.0 * t * H[n] - 2.0 * (double)n * H[n - 1];
}

__device__ __forceinline__ double center(const TreeView& T, int node, int k) {
  return 0.5 * ((double)T.lo[(size_t)node * T.d + k] + (double)T.hi[(size_t)node * T.d + k]);
}

// A box center as an unevaluated float pair hi + lo.  (p - hi) is exact for
// a point p near the center (Sterbenz), so (p - hi) - lo carries only the
// rounding of the difference itself, not the rounding of the center's
// coordinate, which would be an absolute error u |c| -- large against a
// small bandwidth.
struct CenterHL {
  float hi, lo;
};
__device__ __forceinline__ CenterHL center_hl(const TreeView& T, int node, int k) {
  return CenterHL{T.chi[(size_t)node * T.d + k], T.clo[(size_t)node * T.d + k]};
}
__device__ __forceinline__ float minus_center(float p, CenterHL c) { return (p - c.hi) - c.lo; }

template <int D>
__device__ __forceinline__ void load_point(const float* __restrict__ p, float* v) {
  if constexpr (D == 1) {
    v[0] = __ldg(p);
  } else if constexpr (D == 2) {
    const float2 a = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = a.x; v[1] = a.y;
  } else if constexpr (D <= 4) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z;
    if constexpr (D == 4) v[3] = a.w;
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = __ldg(p + k);
  }
}

// ------------------------------------------------------------------ base
// DFGTBase: exact sums over the listed node pairs.
//
// The list is sorted by (bandwidth, query node) with a counting sort, and
// each warp takes a chunk of kBaseChunk consecutive sorted entries, so the
// entries of one query node mostly share a warp: the queries stay in
// registers across them and each query receives one float64 atomic add per
// run of entries instead of one per pair.  The chunk's descriptors are
// loaded in one round trip (one per lane) and broadcast with shuffles.
//
// Reference points are staged per warp in shared memory, negated, as
// structure-of-arrays tiles of kTile points, so one 64-bit load yields the
// coordinate of two consecutive references and every FP32 step works on
// two interactions at once (packed f32x2 add / fma / mul).  Per pair of
// interactions that is 2D+2 packed ops and two SFU ex2, so the kernel is
// bound by the ex2 rate rather than by instruction issue.  For |Q| < 32 the
// warp is split into 32/g lane groups (g = |Q| rounded up to a power of
// two) that share the queries and divide the reference pairs.  A run of
// one reference node is summed in float32; runs are added with Kahan
// compensation and lane groups are combined in float64.

constexpr int kBaseChunk = 8;
constexpr int kNodeBits = 27;  // node indices stay below 2^27 (checked by the tree build)
constexpr int kNodeMask = (1 << kNodeBits) - 1;
constexpr float kFarNeg = -1.0e18f;  // padding point: contributes exp(-huge) = 0

// Counting sort of a pair list by (bandwidth, query node).  Pair and Action
// records share the layout {q, r, h, w}; the sorted value packs r with the
// fourth field w (order p of an action, 0 for a base pair) as r | w << 27.
__global__ void k_sort_count(const Pair* __restrict__ list, int n, int nnQ, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Pair p = list[i];
  atomicAdd(&cnt[(size_t)p.h * nnQ + p.q], 1);
}

__global__ void k_sort_scatter(const Pair* __restrict__ list, int n, int nnQ, int* __restrict__ cursor,
                               int* __restrict__ vsorted, int* __restrict__ ksorted) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Pair p = list[i];
  const int key = p.h * nnQ + p.q;
  const int pos = atomicAdd(&cursor[key], 1);
  vsorted[pos] = p.r | (p.flags << kNodeBits);
  ksorted[pos] = key;
}

// Lane-group width g (a power of two <= 32) for a run of |Q| queries and
// `tot` references when every lane holds two queries: a pass covers 2g
// queries and each lane walks tot / (2 * 32/g) reference pairs; a pass
// also costs a fixed overhead (query set-up, reduction, atomics) worth
// about kPassCost pair iterations.  Pick the g of least modelled cost.
constexpr int kPassCost = 16;
__device__ __forceinline__ int pick_group(int qn, int tot) {
  const int pairs = (tot + 1) / 2;
  int best = 32, cost = 1 << 30;
  for (int g = 32; g >= 1; g >>= 1) {
    const int passes = (qn + 2 * g - 1) / (2 * g);
    const int iters = (pairs + (32 / g) - 1) / (32 / g);
    const int c = passes * (iters + kPassCost);
    if (c < cost) { cost = c; best = g; }
  }
  return best;
}

// Binomial coefficients C(b, a), b, a < 8.
__constant__ float c_binom[8][8] = {
    {1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {1.0f, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {1.0f, 2.0f, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {1.0f, 3.0f, 3.0f, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {1.0f, 4.0f, 6.0f, 4.0f, 1.0f, 0.0f, 0.0f, 0.0f},
    {1.0f, 5.0f, 10.0f, 10.0f, 5.0f, 1.0f, 0.0f, 0.0f},
    {1.0f, 6.0f, 15.0f, 20.0f, 15.0f, 6.0f, 1.0f, 0.0f},
    {1.0f, 7.0f, 21.0f, 35.0f, 35.0f, 21.0f, 7.0f, 1.0f}};
__device__ __forceinline__ float binom_f(int b, int a) { return c_binom[b][a]; }

// Kahan step of a float32 running sum.
__device__ __forceinline__ void kahan_add(float& S, float& C, float v) {
  const float y = v - C;
  const float t = S + y;
  C = (t - S) - y;
  S = t;
}

// One lane's share of a staged tile: reference pairs jp = 2*gid, 2*gid + step, ...
// (step = 2 * number of lane groups) against the lane's two queries a and b.
// EXP selects the expanded form (qa/qb hold W, aa/ab hold A) or the direct
// form (qa/qb hold the query).  Runs of 16 pairs are Kahan-compensated.
template <int D, bool EXP, int TILE>
__device__ __forceinline__ void base_tile_sums(const float (*sR)[TILE], int tn2, int gid, int step,
                                               const float2* qa, const float2* qb, float2 aa, float2 ab,
                                               float2 c2p, float& Sa, float& Ca, float& Sb, float& Cb) {
  for (int jr = 2 * gid; jr < tn2; jr += 16 * step) {
    const int je = min(jr + 16 * step, tn2);
    float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int jp = jr; jp < je; jp += step) {
      float2 rr[D + 1];
#pragma unroll
      for (int k = 0; k < (EXP ? D + 1 : D); ++k) rr[k] = *reinterpret_cast<const float2*>(&sR[k][jp]);
      float2 xa, xb;
      if constexpr (EXP) {
        xa = __fadd2_rn(aa, rr[D]);
        xb = __fadd2_rn(ab, rr[D]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          xa = __ffma2_rn(qa[k], rr[k], xa);
          xb = __ffma2_rn(qb[k], rr[k], xb);
        }
      } else {
        float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float2 ta = __fadd2_rn(qa[k], rr[k]);
          const float2 tb = __fadd2_rn(qb[k], rr[k]);
          da = __ffma2_rn(ta, ta, da);
          db = __ffma2_rn(tb, tb, db);
        }
        xa = __fmul2_rn(da, c2p);
        xb = __fmul2_rn(db, c2p);
      }
      pa = __fadd2_rn(pa, make_float2(ex2_approx(xa.x), ex2_approx(xa.y)));
      pb = __fadd2_rn(pb, make_float2(ex2_approx(xb.x), ex2_approx(xb.y)));
    }
    kahan_add(Sa, Ca, pa.x + pa.y);
    kahan_add(Sb, Cb, pb.x + pb.y);
  }
}

// References staged per warp: D+1 rows of as many points as 48 KB of
// shared memory per block allows.
template <int D>
constexpr int base_tile() {
  return ((48 * 1024 / 4 / kWarpsPerBlock) / (D + 1)) & ~1;
}

// Two forms of the exponent x = c |q - r|^2, c = -log2(e)/(2h^2):
//  * direct: differences q - r, D packed add + D packed fma per pair of
//    references; rounding changes a term by at most (D+3) u x relative;
//  * expanded about the query node's center m, with q~ = q - m, r~ = r - m:
//    x = A_q + B_r + sum_k W_qk r~_k, A_q = c|q~|^2, W_q = -2c q~, B_r = c|r~|^2
//    staged with the reference; one packed add + D packed fma per pair.
//    Its rounding error in x is at most (D+3) u |c| (|q~| + |r~|)^2, the
//    same for every term, so a run uses it only when that bound, taken over
//    the query box and the farthest corner of every reference box, is at
//    most kExpandedErr relative; otherwise the direct form.
constexpr float kExpandedErr = 5e-6f;

template <int D>
__global__ void __launch_bounds__(kT, 3) k_base(TreeView Q, TreeView R, const int* __restrict__ rsorted,
                                             const int* __restrict__ ksorted, int n,
                                             const float* __restrict__ c2v,
                                             const float* __restrict__ inv2h2_up,
                                             double* __restrict__ gacc) {
  constexpr int TILE = base_tile<D>();
  __shared__ __align__(16) float sR[kWarpsPerBlock][D + 1][TILE];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long i0 = ((long)blockIdx.x * kWarpsPerBlock + wib) * kBaseChunk;
  if (i0 >= n) return;
  const int m = (int)min((long)kBaseChunk, n - i0);
  int my_key = -1, my_r = 0, my_rb = 0, my_rn = 0;
  if (lane < m) {
    my_key = ksorted[i0 + lane];
    my_r = rsorted[i0 + lane] & kNodeMask;
    my_rb = R.beg[my_r];
    my_rn = R.cnt[my_r];
  }
  int t = 0;
  while (t < m) {
    // a run: consecutive entries of the same (bandwidth, query node)
    const int key = __shfl_sync(0xffffffffu, my_key, t);
    int e = t + 1;
    while (e < m && __shfl_sync(0xffffffffu, my_key, e) == key) ++e;
    int tot = 0;
    for (int u = t; u < e; ++u) tot += __shfl_sync(0xffffffffu, my_rn, u);
    const int hidx = key / Q.nn, q = key % Q.nn;
    const float c2 = c2v[hidx];
    const int qb = Q.beg[q], qn = Q.cnt[q];
    const int g = pick_group(qn, tot);
    const int ngrp = 32 / g, ql = lane % g, gid = lane / g;
    // expansion center and the error test of the expanded form
    float mc[D];
    float rhoQ2 = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float lo = Q.lo[(size_t)q * D + k], hi = Q.hi[(size_t)q * D + k];
      mc[k] = 0.5f * (lo + hi);
      const float w = fmaxf(__fsub_ru(hi, mc[k]), __fsub_ru(mc[k], lo));
      rhoQ2 = __fmaf_ru(w, w, rhoQ2);
    }
    float far2 = 0.f;  // farthest reference-box corner from mc, squared
    if (lane >= t && lane < e) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float lo = R.lo[(size_t)my_r * D + k], hi = R.hi[(size_t)my_r * D + k];
        const float w = fmaxf(fabsf(__fsub_ru(hi, mc[k])), fabsf(__fsub_rd(lo, mc[k])));
        far2 = __fmaf_ru(w, w, far2);
      }
    }
    for (int o = 16; o > 0; o >>= 1) far2 = fmaxf(far2, __shfl_xor_sync(0xffffffffu, far2, o));
    const float span = __fadd_ru(__fsqrt_ru(rhoQ2), __fsqrt_ru(far2));
    const bool expanded =
        (float)(D + 3) * 5.9604645e-08f * span * span * inv2h2_up[hidx] <= kExpandedErr;
    // Stage references [j0, j0 + tn) of the run's concatenated point list,
    // padded with a far point to an even count; entry by entry.
    auto stage = [&](int j0, int tn) {
      const int tn2 = (tn + 1) & ~1;
      __syncwarp();
      int base = 0;
      for (int u = t; u < e; ++u) {
        const int rn_u = __shfl_sync(0xffffffffu, my_rn, u);
        const int rb_u = __shfl_sync(0xffffffffu, my_rb, u);
        const int lo = max(j0 - base, 0), hi = min(j0 + tn - base, rn_u);
        for (int jj = lo + lane; jj < hi; jj += 32) {
          float rv[D];
          load_point<D>(R.pts + (size_t)(rb_u + jj) * R.dp, rv);
          const int j = base + jj - j0;
          if (expanded) {
            float b2 = 0.f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
              const float rt = rv[k] - mc[k];
              sR[wib][k][j] = rt;
              b2 = fmaf(rt, rt, b2);
            }
            sR[wib][D][j] = c2 * b2;
          } else {
#pragma unroll
            for (int k = 0; k < D; ++k) sR[wib][k][j] = -rv[k];
          }
        }
        base += rn_u;
      }
      if (lane == 0 && tn2 > tn) {
#pragma unroll
        for (int k = 0; k < D; ++k) sR[wib][k][tn] = expanded ? 0.f : kFarNeg;
        sR[wib][D][tn] = -1.0e30f;
      }
      __syncwarp();
      return tn2;
    };
    const bool one_tile = tot <= TILE;
    const int staged2 = one_tile ? stage(0, tot) : 0;
    const float2 c2p = make_float2(c2, c2);
    // every lane holds queries q0 + ql and q0 + g + ql
    for (int q0 = 0; q0 < qn; q0 += 2 * g) {
      const int qia = q0 + ql, qib = q0 + g + ql;
      const bool oka = qia < qn, okb = qib < qn;
      float2 wqa[D], wqb[D], aa, ab;
      {
        float va[D], vb[D];
        if (oka) load_point<D>(Q.pts + (size_t)(qb + qia) * Q.dp, va);
        else
#pragma unroll
          for (int k = 0; k < D; ++k) va[k] = mc[k];
        if (okb) load_point<D>(Q.pts + (size_t)(qb + qib) * Q.dp, vb);
        else
#pragma unroll
          for (int k = 0; k < D; ++k) vb[k] = mc[k];
        float a2 = 0.f, b2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float ta = va[k] - mc[k], tb = vb[k] - mc[k];
          a2 = fmaf(ta, ta, a2);
          b2 = fmaf(tb, tb, b2);
          const float wa = expanded ? -2.f * c2 * ta : va[k];
          const float wb = expanded ? -2.f * c2 * tb : vb[k];
          wqa[k] = make_float2(wa, wa);
          wqb[k] = make_float2(wb, wb);
        }
        aa = make_float2(c2 * a2, c2 * a2);
        ab = make_float2(c2 * b2, c2 * b2);
      }
      float Sa = 0.f, Ca = 0.f, Sb = 0.f, Cb = 0.f;
      for (int j0 = 0; j0 < tot; j0 += TILE) {
        const int tn2 = one_tile ? staged2 : stage(j0, min(TILE, tot - j0));
        if (expanded)
          base_tile_sums<D, true, TILE>(sR[wib], tn2, gid, 2 * ngrp, wqa, wqb, aa, ab, c2p, Sa, Ca, Sb, Cb);
        else
          base_tile_sums<D, false, TILE>(sR[wib], tn2, gid, 2 * ngrp, wqa, wqb, aa, ab, c2p, Sa, Ca, Sb, Cb);
      }
      float va = Sa - Ca, vb = Sb - Cb;
      for (int o = g; o < 32; o <<= 1) {
        va += __shfl_xor_sync(0xffffffffu, va, o);
        vb += __shfl_xor_sync(0xffffffffu, vb, o);
      }
      if (gid == 0 && oka) atomicAdd(&gacc[(size_t)hidx * Q.n + qb + qia], (double)va);
      if (gid == 0 && okb) atomicAdd(&gacc[(size_t)hidx * Q.n + qb + qib], (double)vb);
    }
    t = e;
  }
}

// D >= 6: the same chunked walk with runtime dimension and scalar math.
__global__ void __launch_bounds__(kT) k_base_g(TreeView Q, TreeView R, const int* __restrict__ rsorted,
                                               const int* __restrict__ ksorted, int n,
                                               const double* __restrict__ hv,
                                               double* __restrict__ gacc) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long i0 = ((long)blockIdx.x * kWarpsPerBlock + wib) * kBaseChunk;
  if (i0 >= n) return;
  const int m = (int)min((long)kBaseChunk, n - i0);
  const int d = Q.d;
  for (int u = 0; u < m; ++u) {
    const int key = ksorted[i0 + u], r = rsorted[i0 + u] & kNodeMask;
    const int hidx = key / Q.nn, q = key % Q.nn;
    const double h = hv[hidx];
    const float c2 = (float)(-kLog2e / (2.0 * h * h));
    const int qb = Q.beg[q], qn = Q.cnt[q], rb = R.beg[r], rn = R.cnt[r];
    for (int qi = lane; qi < qn; qi += 32) {
      float qv[kMaxD];
#pragma unroll
      for (int k = 0; k < kMaxD; ++k) qv[k] = k < d ? Q.pts[(size_t)(qb + qi) * Q.dp + k] : 0.f;
      float part = 0.f;
      for (int j = 0; j < rn; ++j) {
        float d2 = 0.f;
#pragma unroll
        for (int k = 0; k < kMaxD; ++k) {
          if (k < d) {
            const float tt = qv[k] - R.pts[(size_t)(rb + j) * R.dp + k];
            d2 = fmaf(tt, tt, d2);
          }
        }
        part += ex2_approx(d2 * c2);
      }
      atomicAdd(&gacc[(size_t)hidx * Q.n + qb + qi], (double)part);
    }
  }
}

// Scaled far-field moments M_alpha = m_alpha (2h^2)^(-|alpha|/2) for alpha < p
// (zero elsewhere) into shared memory, float32.
template <int D, int PM, int P>
__device__ __forceinline__ void stage_moments(const float* __restrict__ mn, float ws, int p, float* Ms,
                                              int lane) {
  // M_alpha = m~_alpha (w s)^|alpha| for alpha < p, 0 elsewhere (float32)
  for (int idx = lane; idx < P; idx += 32) {
    int ab = 0;
    bool ok = true;
    {
      int v = idx;
#pragma unroll
      for (int k = D - 1; k >= 0; --k) { const int a = v % PM; v /= PM; ab += a; ok = ok && a < p; }
    }
    Ms[idx] = ok ? mn[idx] * pow_int_f(ws, ab) : 0.f;
  }
}

// ------------------------------------------------------------- far field
// EvaluateFarFieldExpansion: sum_{alpha<p} M_alpha h_alpha((q - R.c)/sqrt(2h^2)).
template <int D>
__global__ void __launch_bounds__(kT) k_farfield(TreeView Q, TreeView R,
                                                 const Action* __restrict__ list, int n,
                                                 const float* __restrict__ sfv,
                                                 double* __restrict__ gacc) {
  constexpr int PM = pmax_of(D);
  constexpr int P = ipow_c(PM, D);
  __shared__ float sM[kWarpsPerBlock][P];
  const int wib = threadIdx.x >> 5;
  const int w = blockIdx.x * kWarpsPerBlock + wib;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const Action a = list[w];
  const float sf = sfv[a.h];
  float* Ms = sM[wib];
  stage_moments<D, PM, P>(R.mnorm + (size_t)a.r * P, R.whalf[a.r] * sf, a.p, Ms, lane);
  __syncwarp();
  CenterHL cR[D];
#pragma unroll
  for (int k = 0; k < D; ++k) cR[k] = center_hl(R, a.r, k);
  const int qb = Q.beg[a.q], qn = Q.cnt[a.q];
  for (int qi = lane; qi < qn; qi += 32) {
    float qv[D];
    load_point<D>(Q.pts + (size_t)(qb + qi) * Q.dp, qv);
    float H[D][PM];
#pragma unroll
    for (int k = 0; k < D; ++k) hermite_f32<PM>(minus_center(qv[k], cR[k]) * sf, H[k]);
    float acc = 0.f;
#pragma unroll
    for (int idx = 0; idx < P; ++idx) {
      float t = Ms[idx];
#pragma unroll
      for (int k = 0; k < D; ++k) t *= H[k][digit_c<D, PM>(idx, k)];
      acc += t;
    }
    atomicAdd(&gacc[(size_t)a.h * Q.n + qb + qi], (double)acc);
  }
}

// ------------------------------------------------------------ direct local
// AccumulateDirectLocalMoment:
// L_beta(Q) += ((-1)^{|beta|}/beta!) sum_{r in R} h_beta((Q.c - r)/sqrt(2h^2)).
// The list is sorted by (bandwidth, query node) like the base case, and a
// warp takes kBaseChunk consecutive sorted entries: every run of one query
// node accumulates its coefficients in registers (lane per coefficient
// position) and adds them to L once.  For each batch of 32 reference points
// each lane tabulates the 1-D Hermite functions of one point in shared
// memory, then every lane sums its coefficient over the batch; batches are
// summed in float32 and added in float64.  An entry of order p contributes
// only to beta < p.
template <int D>
__global__ void __launch_bounds__(kT) k_local(TreeView Q, TreeView R, const int* __restrict__ rsorted,
                                              const int* __restrict__ ksorted, int n,
                                              const float* __restrict__ sfv,
                                              double* __restrict__ L, int* __restrict__ pused) {
  constexpr int PM = pmax_of(D);
  constexpr int P = ipow_c(PM, D);
  constexpr int S = (P + 31) / 32;
  __shared__ float sH[kWarpsPerBlock][32][D][PM];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long i0 = ((long)blockIdx.x * kWarpsPerBlock + wib) * kBaseChunk;
  if (i0 >= n) return;
  const int m = (int)min((long)kBaseChunk, n - i0);
  int my_key = -1, my_r = 0, my_p = 0;
  if (lane < m) {
    my_key = ksorted[i0 + lane];
    const int v = rsorted[i0 + lane];
    my_r = v & kNodeMask;
    my_p = v >> kNodeBits;
  }
  int al[S][D];
  double fsign[S];
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    int v = lane + 32 * sl, ab = 0;
    double f = 1.0;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) { al[sl][k] = v % PM; v /= PM; ab += al[sl][k]; f *= fact_d(al[sl][k]); }
    fsign[sl] = ((ab & 1) ? -1.0 : 1.0) / f;
  }
  int t = 0;
  while (t < m) {
    const int key = __shfl_sync(0xffffffffu, my_key, t);
    int e = t + 1;
    while (e < m && __shfl_sync(0xffffffffu, my_key, e) == key) ++e;
    const int hidx = key / Q.nn, q = key % Q.nn;
    const float sf = sfv[hidx];
    CenterHL cQ[D];
#pragma unroll
    for (int k = 0; k < D; ++k) cQ[k] = center_hl(Q, q, k);
    float accS[S], accC[S];
#pragma unroll
    for (int sl = 0; sl < S; ++sl) accS[sl] = accC[sl] = 0.f;
    int prun = 0;
    for (int u = t; u < e; ++u) {
      const int r = __shfl_sync(0xffffffffu, my_r, u);
      const int p = __shfl_sync(0xffffffffu, my_p, u);
      prun = max(prun, p);
      const int rb = R.beg[r], rn = R.cnt[r];
      for (int j0 = 0; j0 < rn; j0 += 32) {
        const int j = j0 + lane;
        if (j < rn) {
          float rv[D];
          load_point<D>(R.pts + (size_t)(rb + j) * R.dp, rv);
#pragma unroll
          for (int k = 0; k < D; ++k) hermite_f32<PM>(-minus_center(rv[k], cQ[k]) * sf, sH[wib][lane][k]);
        } else {
#pragma unroll
          for (int k = 0; k < D; ++k)
#pragma unroll
            for (int e2 = 0; e2 < PM; ++e2) sH[wib][lane][k][e2] = 0.f;
        }
        __syncwarp();
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
          const int idx = lane + 32 * sl;
          bool ok = idx < P;
#pragma unroll
          for (int k = 0; k < D; ++k) ok = ok && al[sl][k] < p;
          if (ok) {
            float part = 0.f;
            for (int jj = 0; jj < 32; ++jj) {
              float tt = sH[wib][jj][0][al[sl][0]];
#pragma unroll
              for (int k = 1; k < D; ++k) tt *= sH[wib][jj][k][al[sl][k]];
              part += tt;
            }
            kahan_add(accS[sl], accC[sl], part);
          }
        }
        __syncwarp();
      }
    }
    const size_t hq = (size_t)hidx * Q.nn + q;
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      const int idx = lane + 32 * sl;
      const double v = (double)accS[sl] - (double)accC[sl];
      if (idx < P && v != 0.0) atomicAdd(&L[hq * P + idx], v * fsign[sl]);
    }
    if (lane == 0) atomicMax(&pused[hq], prun);
    t = e;
  }
}

// --------------------------------------------------------- far to local
// TransFarToLocal (Lemma 3.3, Eq. farfield_to_local_formula):
// L_beta(Q) += ((-1)^{|beta|}/beta!) sum_{alpha<p} M_alpha h_{alpha+beta}((Q.c - R.c)/sqrt(2h^2)).
// The 1-D Hermite table up to order 2p_max-2 is computed in float64.
template <int D>
__global__ void __launch_bounds__(kT) k_f2l(TreeView Q, TreeView R, const Action* __restrict__ list,
                                            int n, const double* __restrict__ hv,
                                            double* __restrict__ L, int* __restrict__ pused) {
  constexpr int PM = pmax_of(D);
  constexpr int P = ipow_c(PM, D);
  constexpr int NH = 2 * PM - 1;
  constexpr int S = (P + 31) / 32;
  __shared__ float sM[kWarpsPerBlock][P];
  __shared__ float sH[kWarpsPerBlock][D][NH];
  const int wib = threadIdx.x >> 5;
  const int w = blockIdx.x * kWarpsPerBlock + wib;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const Action a = list[w];
  const double h = hv[a.h];
  const double s = 1.0 / sqrt(2.0 * h * h);
  if (lane < D) {
    double H[NH];
    hermite_f64<NH>((center(Q, a.q, lane) - center(R, a.r, lane)) * s, H);
#pragma unroll
    for (int e = 0; e < NH; ++e) sH[wib][lane][e] = (float)H[e];
  }
  stage_moments<D, PM, P>(R.mnorm + (size_t)a.r * P, R.whalf[a.r] * (float)s, a.p, sM[wib], lane);
  __syncwarp();
  const size_t hq = (size_t)a.h * Q.nn + a.q;
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    const int idx = lane + 32 * sl;
    if (idx >= P) break;
    int be[D];
    int ab = 0;
    bool ok = true;
    double f = 1.0;
    {
      int v = idx;
#pragma unroll
      for (int k = D - 1; k >= 0; --k) { be[k] = v % PM; v /= PM; ab += be[k]; ok = ok && be[k] < a.p; f *= fact_d(be[k]); }
    }
    if (!ok) continue;
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < P; ++j) {
      float t = sM[wib][j];
#pragma unroll
      for (int k = 0; k < D; ++k) t *= sH[wib][k][digit_c<D, PM>(j, k) + be[k]];
      acc += t;
    }
    atomicAdd(&L[hq * P + idx], ((ab & 1) ? -(double)acc : (double)acc) / f);
  }
  if (lane == 0) atomicMax(&pused[hq], a.p);
}

// ------------------------------------------------------------- prune
// Distance-bound prune applied to listed pairs (the traversal applies it
// inline): L_0(Q) += |R| (K(d^l) + K(d^u)) / 2.
__global__ void k_prune_apply(TreeView Q, TreeView R, const Pair* __restrict__ list, int n,
                              const float* __restrict__ inv2h2_dn, const float* __restrict__ inv2h2_up,
                              double* __restrict__ L, int* __restrict__ pused) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Pair pr = list[i];
  float dl2, du2, sq, sr;
  box_geometry<0>(Q, pr.q, R, pr.r, dl2, du2, sq, sr);
  const float Kl = kernel_upper(dl2, inv2h2_dn[pr.h]);
  const float Ku = kernel_lower(du2, inv2h2_up[pr.h]);
  const size_t hq = (size_t)pr.h * Q.nn + pr.q;
  atomicAdd(&L[hq * Q.P], (double)(0.5f * (float)R.cnt[pr.r]) * ((double)Kl + (double)Ku));
  atomicMax(&pused[hq], 1);
}

// ---------------------------------------------------------------- post
// DFGTPost, fused.  The paper shifts every local expansion down the query
// tree with TransLocalToLocal (Lemma 3.6) and reads the leaves out with
// EvaluateLocalExpansion.  Re-centering a polynomial is exact, so shifting
// each expansion of a leaf's ancestors straight to the leaf's center gives
// the same polynomial as the level-by-level pass; one warp per leaf does
// that for every bandwidth, sums the shifted coefficients (Kahan-
// compensated float32; the constant term in float64), evaluates the sum
// at the leaf's points and adds the exact and far-field parts, writing G
// in the caller's query order.  One launch instead of one per level.
//
// Shift from center c to c' along one dimension, d = (c' - c)/sqrt(2h^2):
// L'_a = sum_{a<=b<p} C(b, a) d^{b-a} L_b; the D dimensions are applied one
// after the other (D p^D p operations).  Every shifted coefficient is a sum
// of terms whose absolute values add up, at a point x of the leaf, to at
// most sum_alpha |L_alpha| prod_k (w_k s)^alpha_k with w the half sides of
// the ancestor's box (|x - c'| + |c' - c| <= w per dimension for nested
// boxes), the same quantity that bounds the expansion's own evaluation; the
// float32 rounding of a shift is at most 6 p D u times it (the rounded
// d carries 4u, its powers up to 4(p-1)u, Horner's rule (2p-1)u per
// dimension), which the rounding allowance of the truncation bounds
// includes.
constexpr int kMaxDepth = 128;

template <int D>
__global__ void __launch_bounds__(kT) k_post(TreeView Q, const int* __restrict__ leaves, int nleaves,
                                             const double* __restrict__ gacc,
                                             const double* __restrict__ L,
                                             const int* __restrict__ pused,
                                             const float* __restrict__ sfv, int nh,
                                             double* __restrict__ G) {
  constexpr int PM = pmax_of(D);
  constexpr int P = ipow_c(PM, D);
  constexpr int S = (P + 31) / 32;
  __shared__ int sPath[kWarpsPerBlock][kMaxDepth];
  __shared__ float sT[kWarpsPerBlock][2][P];
  __shared__ float sA[kWarpsPerBlock][P];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = blockIdx.x * kWarpsPerBlock + wib;
  if (li >= nleaves) return;
  const int leaf = leaves[li];
  int len = 0;
  if (lane == 0) {
    for (int v = leaf; v >= 0 && len < kMaxDepth; v = Q.parent[v]) sPath[wib][len++] = v;
  }
  len = __shfl_sync(0xffffffffu, len, 0);
  __syncwarp();
  CenterHL cl[D];
#pragma unroll
  for (int k = 0; k < D; ++k) cl[k] = center_hl(Q, leaf, k);
  const int qb = Q.beg[leaf], qn = Q.cnt[leaf];
  for (int hidx = 0; hidx < nh; ++hidx) {
    const float sf = sfv[hidx];
    float accS[S], accC[S];
#pragma unroll
    for (int sl = 0; sl < S; ++sl) accS[sl] = accC[sl] = 0.f;
    double c0 = 0.0;  // constant term, the same in every lane
    int pa = 0;       // highest order on the path
    for (int i0 = 0; i0 < len; i0 += 32) {
      const int node = i0 + lane < len ? sPath[wib][i0 + lane] : -1;
      const int pu = node >= 0 ? pused[(size_t)hidx * Q.nn + node] : 0;
      unsigned m = __ballot_sync(0xffffffffu, pu > 0);
      while (m) {
        const int bl = __ffs(m) - 1;
        m &= m - 1;
        const int j = __shfl_sync(0xffffffffu, node, bl);
        const int pj = __shfl_sync(0xffffffffu, pu, bl);
        const double* Lj = L + ((size_t)hidx * Q.nn + j) * P;
        c0 += Lj[0];
        pa = max(pa, pj);
        if (pj == 1) continue;  // a constant shifts unchanged
        // the non-constant part, shifted from c_j to the leaf's center
        for (int idx = lane; idx < P; idx += 32) sT[wib][0][idx] = idx == 0 ? 0.f : (float)Lj[idx];
        __syncwarp();
        int cur = 0;
        if (j != leaf) {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const CenterHL cj = center_hl(Q, j, k);
            const float dk = ((cl[k].hi - cj.hi) + (cl[k].lo - cj.lo)) * sf;
            const int stride = ipow_c(PM, D - 1 - k);
            for (int idx = lane; idx < P; idx += 32) {
              const int ak = (idx / stride) % PM;
              float acc = 0.f;
              if (ak < pj) {
                // sum_{b=ak}^{pj-1} C(b, ak) d^(b-ak) L_b, Horner in d
                for (int bk = pj - 1; bk >= ak; --bk)
                  acc = fmaf(acc, dk, binom_f(bk, ak) * sT[wib][cur][idx + (bk - ak) * stride]);
              }
              sT[wib][cur ^ 1][idx] = acc;
            }
            __syncwarp();
            cur ^= 1;
          }
        }
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
          const int idx = lane + 32 * sl;
          if (idx < P) kahan_add(accS[sl], accC[sl], sT[wib][cur][idx]);
        }
        __syncwarp();
      }
    }
    // coefficients of the summed expansion at the leaf's center
    double cst = c0;
    if (pa > 1) {
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        const int idx = lane + 32 * sl;
        if (idx < P) sA[wib][idx] = idx == 0 ? 0.f : accS[sl] - accC[sl];
      }
      cst += (double)__shfl_sync(0xffffffffu, accS[0] - accC[0], 0);
      __syncwarp();
    }
    for (int pi = lane; pi < qn; pi += 32) {
      const int i = qb + pi;
      double val = gacc[(size_t)hidx * Q.n + i] + cst;
      if (pa > 1) {
        float qv[D];
        load_point<D>(Q.pts + (size_t)i * Q.dp, qv);
        float X[D][PM];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float x = minus_center(qv[k], cl[k]) * sf;
          float v = 1.f;
#pragma unroll
          for (int e = 0; e < PM; ++e) { X[k][e] = v; v *= x; }
        }
        float acc = 0.f;
#pragma unroll
        for (int idx = 1; idx < P; ++idx) {
          if (!below_c<D, PM>(idx, pa)) continue;
          float term = sA[wib][idx];
#pragma unroll
          for (int k = 0; k < D; ++k) term *= X[k][digit_c<D, PM>(idx, k)];
          acc += term;
        }
        val += (double)acc;
      }
      G[(size_t)hidx * Q.n + Q.perm[i]] = val;
    }
    __syncwarp();
  }
}

// ------------------------------------------------- order 0 (D >= 6)
// With p_max = 1 every expansion keeps only its alpha = 0 term:
// F: |R| e^{-||q-R.c||^2/2h^2};  D: L_0 += sum_r e^{-||Q.c-r||^2/2h^2};
// T: L_0 += |R| e^{-||Q.c-R.c||^2/2h^2}.
__global__ void __launch_bounds__(kT) k_farfield_g(TreeView Q, TreeView R, const Action* __restrict__ list,
                                                   int n, const double* __restrict__ hv,
                                                   double* __restrict__ gacc) {
  const int w = (blockIdx.x * kT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const Action a = list[w];
  const double h = hv[a.h];
  const float c2 = (float)(-kLog2e / (2.0 * h * h));
  const float m0 = R.mnorm[a.r];
  const int qb = Q.beg[a.q], qn = Q.cnt[a.q];
  for (int qi = lane; qi < qn; qi += 32) {
    float d2 = 0.f;
    for (int k = 0; k < Q.d; ++k) {
      const float t = minus_center(Q.pts[(size_t)(qb + qi) * Q.dp + k], center_hl(R, a.r, k));
      d2 = fmaf(t, t, d2);
    }
    atomicAdd(&gacc[(size_t)a.h * Q.n + qb + qi], (double)(m0 * ex2_approx(d2 * c2)));
  }
}

__global__ void __launch_bounds__(kT) k_local_g(TreeView Q, TreeView R, const Action* __restrict__ list,
                                                int n, const double* __restrict__ hv,
                                                double* __restrict__ L, int* __restrict__ pused) {
  const int w = (blockIdx.x * kT + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const Action a = list[w];
  const double h = hv[a.h];
  const float c2 = (float)(-kLog2e / (2.0 * h * h));
  const int rb = R.beg[a.r], rn = R.cnt[a.r];
  float part = 0.f;
  for (int j = lane; j < rn; j += 32) {
    float d2 = 0.f;
    for (int k = 0; k < Q.d; ++k) {
      const float t = minus_center(R.pts[(size_t)(rb + j) * R.dp + k], center_hl(Q, a.q, k));
      d2 = fmaf(t, t, d2);
    }
    part += ex2_approx(d2 * c2);
  }
  double v = part;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const size_t hq = (size_t)a.h * Q.nn + a.q;
  if (lane == 0) {
    atomicAdd(&L[hq], v);
    atomicMax(&pused[hq], 1);
  }
}

__global__ void k_f2l_g(TreeView Q, TreeView R, const Action* __restrict__ list, int n,
                        const double* __restrict__ hv, double* __restrict__ L,
                        int* __restrict__ pused) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Action a = list[i];
  const double h = hv[a.h];
  double d2 = 0.0;
  for (int k = 0; k < Q.d; ++k) {
    const double t = center(Q, a.q, k) - center(R, a.r, k);
    d2 += t * t;
  }
  const size_t hq = (size_t)a.h * Q.nn + a.q;
  atomicAdd(&L[hq], R.mom[a.r] * exp(-d2 / (2.0 * h * h)));
  atomicMax(&pused[hq], 1);
}

// D >= 6: only constants, summed along the path from the root.
__global__ void __launch_bounds__(kT) k_post_g(TreeView Q, const int* __restrict__ leaves, int nleaves,
                                               const double* __restrict__ gacc,
                                               const double* __restrict__ L,
                                               const int* __restrict__ pused, int nh,
                                               double* __restrict__ G) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = blockIdx.x * kWarpsPerBlock + wib;
  if (li >= nleaves) return;
  const int leaf = leaves[li];
  const int qb = Q.beg[leaf], qn = Q.cnt[leaf];
  for (int hidx = 0; hidx < nh; ++hidx) {
    double c0 = 0.0;
    for (int v = leaf; v >= 0; v = Q.parent[v]) {
      const size_t hv = (size_t)hidx * Q.nn + v;
      if (pused[hv] > 0) c0 += L[hv];
    }
    for (int pi = lane; pi < qn; pi += 32)
      G[(size_t)hidx * Q.n + Q.perm[qb + pi]] = gacc[(size_t)hidx * Q.n + qb + pi] + c0;
  }
}

inline int warp_grid(long items) { return (int)((items * 32 + kT - 1) / kT); }

}  // namespace

#define DISPATCH_D(d, ...)                             \
  switch (d) {                                         \
    case 1: { constexpr int DD = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int DD = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int DD = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int DD = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int DD = 5; __VA_ARGS__; } break; \
    default: break;                                    \
  }

// Sort a list by (bandwidth, query node) into sc: vsorted, ksorted.
static cudaError_t sort_by_query(const Pair* list, int n, int nnQ, int nh, BaseScratch& sc,
                                 cudaStream_t s, long long* launches, int** vs, int** ks) {
  const long nkeys = (long)nh * nnQ;
  cudaError_t e;
  if ((e = sc.cnt->ensure((nkeys + 1) * sizeof(int))) != cudaSuccess) return e;
  if ((e = sc.off->ensure((nkeys + 1) * sizeof(int))) != cudaSuccess) return e;
  if ((e = sc.rsorted->ensure(2 * (size_t)n * sizeof(int))) != cudaSuccess) return e;
  int* cnt = sc.cnt->as<int>();
  int* off = sc.off->as<int>();
  *vs = sc.rsorted->as<int>();
  *ks = *vs + n;
  if ((e = cudaMemsetAsync(cnt, 0, nkeys * sizeof(int), s)) != cudaSuccess) return e;
  k_sort_count<<<(n + kT - 1) / kT, kT, 0, s>>>(list, n, nnQ, cnt);
  if ((e = scan_exclusive(cnt, off, (int)nkeys, *sc.scan_tmp, s, launches)) != cudaSuccess) return e;
  k_sort_scatter<<<(n + kT - 1) / kT, kT, 0, s>>>(list, n, nnQ, off, *vs, *ks);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_base(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                        const Pair* list, int n, BaseScratch& sc, cudaStream_t s, long long* launches) {
  if (n <= 0) return cudaSuccess;
  int *rsorted, *ksorted;
  cudaError_t e = sort_by_query(list, n, Q.nn, b.nh, sc, s, launches, &rsorted, &ksorted);
  if (e != cudaSuccess) return e;
  const long warps = (n + kBaseChunk - 1) / kBaseChunk;
  const int g = (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (Q.d <= 5) {
    DISPATCH_D(Q.d, k_base<DD><<<g, kT, 0, s>>>(Q, R, rsorted, ksorted, n, b.c2, b.inv2h2_up, b.gacc));
  } else {
    k_base_g<<<g, kT, 0, s>>>(Q, R, rsorted, ksorted, n, b.h, b.gacc);
  }
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_farfield(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                            const Action* list, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int g = warp_grid(n);
  if (Q.d <= 5) {
    DISPATCH_D(Q.d, k_farfield<DD><<<g, kT, 0, s>>>(Q, R, list, n, b.sf, b.gacc));
  } else {
    k_farfield_g<<<g, kT, 0, s>>>(Q, R, list, n, b.h, b.gacc);
  }
  return cudaGetLastError();
}

cudaError_t launch_local(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                         const Action* list, int n, BaseScratch& sc, cudaStream_t s,
                         long long* launches) {
  if (n <= 0) return cudaSuccess;
  if (Q.d <= 5) {
    int *vsorted, *ksorted;
    cudaError_t e = sort_by_query(reinterpret_cast<const Pair*>(list), n, Q.nn, b.nh, sc, s, launches,
                                  &vsorted, &ksorted);
    if (e != cudaSuccess) return e;
    const long warps = (n + kBaseChunk - 1) / kBaseChunk;
    const int g = (int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
    DISPATCH_D(Q.d, k_local<DD><<<g, kT, 0, s>>>(Q, R, vsorted, ksorted, n, b.sf, b.L, b.pused));
  } else {
    k_local_g<<<warp_grid(n), kT, 0, s>>>(Q, R, list, n, b.h, b.L, b.pused);
  }
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_f2l(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                       const Action* list, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (Q.d <= 5) {
    const int g = warp_grid(n);
    DISPATCH_D(Q.d, k_f2l<DD><<<g, kT, 0, s>>>(Q, R, list, n, b.h, b.L, b.pused));
  } else {
    k_f2l_g<<<(n + kT - 1) / kT, kT, 0, s>>>(Q, R, list, n, b.h, b.L, b.pused);
  }
  return cudaGetLastError();
}

cudaError_t launch_prune_apply(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                               const Pair* list, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_prune_apply<<<(n + kT - 1) / kT, kT, 0, s>>>(Q, R, list, n, b.inv2h2_dn, b.inv2h2_up, b.L, b.pused);
  return cudaGetLastError();
}

cudaError_t launch_post(const TreeView& Q, const int* leaves, int nleaves, const TravBuffers& b,
                        double* G, cudaStream_t s) {
  if (nleaves <= 0) return cudaSuccess;
  const int g = (nleaves + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (Q.d <= 5) {
    DISPATCH_D(Q.d, k_post<DD><<<g, kT, 0, s>>>(Q, leaves, nleaves, b.gacc, b.L, b.pused, b.sf, b.nh, G));
  } else {
    k_post_g<<<g, kT, 0, s>>>(Q, leaves, nleaves, b.gacc, b.L, b.pused, b.nh, G);
  }
  return cudaGetLastError();
}

}  // namespace dfgt
