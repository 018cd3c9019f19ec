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
#include "base_hd_forms.cuh"
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
// each warp takes kEntryChunk = 32 consecutive sorted entries, one per lane:
// every descriptor of the chunk (reference block, query node, its box,
// the expansion test) is fetched in one round trip and broadcast with
// shuffles.  Consecutive entries of one (bandwidth, query node) form a
// run; its references are processed as one concatenated list, so each
// query of the run receives one float64 atomic add per tile.
//
// References are copied raw into shared memory with cp.async one tile
// ahead (the next tile of the run, or the first tile of the next run)
// while the current tile is summed, so global latency overlaps the SFU
// work.  A staged tile is rewritten once per run into pair-interleaved
// rows: for references j, j+1 the values (x_j, x_j+1, y_j, y_j+1, ...,
// B_j, B_j+1), so two 128-bit shared loads give every operand of a packed
// f32x2 step on two interactions.  Each lane holds two queries; for a run
// of few queries the warp splits into lane groups that share the queries
// and divide the references.
// One warp per block: the warps' work is uneven (runs of any length), and
// a block of several warps holds the slots of its finished warps until
// the slowest is done (one-warp blocks ran the exact sums 2.5% faster).
constexpr int kBaseWarps = 1;     // warps per block of the base case
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
constexpr int kPassCost = 32;  // measured: 4, 8, 16, 32, 64 -> 4.58, 4.32, 4.20, 4.17, 4.21 ms
__device__ __forceinline__ int pick_group(int qn, int tot) {
  const int pairs = (tot + 1) / 2;
  int best = 32, cost = 1 << 30;
  for (int lg = 5; lg >= 0; --lg) {  // g = 2^lg
    const int g = 1 << lg;
    const int passes = (qn + 2 * g - 1) >> (lg + 1);
    const int iters = (pairs + (32 >> lg) - 1) >> (5 - lg);
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

// Shapes of the base-case tiles for dimension D: RAW floats per staged
// reference (the tree's padded row), PAIRW floats per interleaved
// reference pair (padded to whole float4s), SV float4 per pair slot (room
// for both the two raw rows and the interleaved pair, so a pair is
// rewritten in place) and TILE references per warp.
template <int D>
struct BaseShape {
  static constexpr int RAW = D <= 2 ? D : ((D + 3) & ~3);
  static constexpr int PAIRW = ((2 * (D + 1) + 3) / 4) * 4;
  static constexpr int NV = PAIRW / 4;
  static constexpr int SV = (2 * RAW > PAIRW ? 2 * RAW : PAIRW) / 4;
  static constexpr int TILE = D == 1 ? 1024 : D == 2 ? 512 : D == 3 ? 448 : 192;
  // a tile's reference pairs are padded to a multiple of the lane groups (up to 32)
  static_assert((TILE / 2) % 32 == 0, "TILE / 2 must be a multiple of 32");
};

__device__ __forceinline__ void cp_async_row(float* dst, const float* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const size_t g = __cvta_generic_to_global(src);
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(g) : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(g) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// One interaction pair step: reference pair at p against the lane's two
// queries; adds 2^x of the four interactions to pa / pb.
template <int D, bool EXP>
__device__ __forceinline__ void base_step(const float4* __restrict__ p, const float2* wa, const float2* wb,
                                          float2 c2p, float2& pa, float2& pb) {
  constexpr int NV = BaseShape<D>::NV;
  float f[4 * NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float4 t4 = p[v];
    f[4 * v] = t4.x; f[4 * v + 1] = t4.y; f[4 * v + 2] = t4.z; f[4 * v + 3] = t4.w;
  }
  float2 xa, xb;
  if constexpr (EXP) {
    xa = make_float2(f[2 * D], f[2 * D + 1]);
    xb = xa;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float2 rk = make_float2(f[2 * k], f[2 * k + 1]);
      xa = __ffma2_rn(wa[k], rk, xa);
      xb = __ffma2_rn(wb[k], rk, xb);
    }
  } else {
    float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float2 rk = make_float2(f[2 * k], f[2 * k + 1]);
      const float2 ta = __fadd2_rn(wa[k], rk);
      const float2 tb = __fadd2_rn(wb[k], rk);
      da = __ffma2_rn(ta, ta, da);
      db = __ffma2_rn(tb, tb, db);
    }
    xa = __fmul2_rn(da, c2p);
    xb = __fmul2_rn(db, c2p);
  }
  pa = __fadd2_rn(pa, make_float2(ex2_approx(xa.x), ex2_approx(xa.y)));
  pb = __fadd2_rn(pb, make_float2(ex2_approx(xb.x), ex2_approx(xb.y)));
}

// One lane's share of an interleaved tile: reference pairs jp = gid,
// gid + ngrp, ... against the lane's two queries a and b.  EXP selects the
// expanded form (wa/wb hold W_q; the exponent is B_r + W_q . r~, A_q is
// applied by the caller) or the direct form (wa/wb hold the query, rows
// the negated reference).  Blocks of 16 steps (unrolled, no bounds tests)
// are summed in float32 and added with Kahan compensation.
template <int D, bool EXP>
__device__ __forceinline__ void base_tile_sums(const float4* __restrict__ T, int np2, int gid, int ngrp,
                                               const float2* wa, const float2* wb, float2 c2p,
                                               float& Sa, float& Ca, float& Sb, float& Cb) {
  // np2 is padded to a multiple of ngrp (a power of two): the same count in every lane
  int left = np2 >> (31 - __clz(ngrp));
  constexpr int SV = BaseShape<D>::SV;
  const float4* p = T + gid * SV;
  const int stride = ngrp * SV;
  for (; left >= 16; left -= 16) {
    float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      base_step<D, EXP>(p, wa, wb, c2p, pa, pb);
      p += stride;
    }
    kahan_add(Sa, Ca, pa.x + pa.y);
    kahan_add(Sb, Cb, pb.x + pb.y);
  }
  if (left > 0) {
    float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
    for (; left >= 4; left -= 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        base_step<D, EXP>(p, wa, wb, c2p, pa, pb);
        p += stride;
      }
    }
    for (; left > 0; --left) {
      base_step<D, EXP>(p, wa, wb, c2p, pa, pb);
      p += stride;
    }
    kahan_add(Sa, Ca, pa.x + pa.y);
    kahan_add(Sb, Cb, pb.x + pb.y);
  }
}

// Direct form with the self interaction left out (leave-one-out sums over
// one tree): the pair slot carries the two references' point indices after
// their coordinates, and a query meets its own index with weight 0.
template <int D>
__device__ __forceinline__ void base_step_loo(const float4* __restrict__ p, const float2* wa, const float2* wb,
                                              float2 c2p, int ia, int ib, float2& pa, float2& pb) {
  constexpr int NV = BaseShape<D>::NV;
  float f[4 * NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float4 t4 = p[v];
    f[4 * v] = t4.x; f[4 * v + 1] = t4.y; f[4 * v + 2] = t4.z; f[4 * v + 3] = t4.w;
  }
  float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float2 rk = make_float2(f[2 * k], f[2 * k + 1]);
    const float2 ta = __fadd2_rn(wa[k], rk);
    const float2 tb = __fadd2_rn(wb[k], rk);
    da = __ffma2_rn(ta, ta, da);
    db = __ffma2_rn(tb, tb, db);
  }
  const float2 xa = __fmul2_rn(da, c2p), xb = __fmul2_rn(db, c2p);
  const int r0 = __float_as_int(f[2 * D]), r1 = __float_as_int(f[2 * D + 1]);
  pa = __fadd2_rn(pa, make_float2(ia == r0 ? 0.f : ex2_approx(xa.x), ia == r1 ? 0.f : ex2_approx(xa.y)));
  pb = __fadd2_rn(pb, make_float2(ib == r0 ? 0.f : ex2_approx(xb.x), ib == r1 ? 0.f : ex2_approx(xb.y)));
}

template <int D>
__device__ __forceinline__ void base_tile_sums_loo(const float4* __restrict__ T, int np2, int gid, int ngrp,
                                                   const float2* wa, const float2* wb, float2 c2p, int ia, int ib,
                                                   float& Sa, float& Ca, float& Sb, float& Cb) {
  constexpr int SV = BaseShape<D>::SV;
  int left = np2 >> (31 - __clz(ngrp));
  const float4* p = T + gid * SV;
  const int stride = ngrp * SV;
  while (left > 0) {
    float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
    const int nb = left < 16 ? left : 16;
    for (int u = 0; u < nb; ++u) {
      base_step_loo<D>(p, wa, wb, c2p, ia, ib, pa, pb);
      p += stride;
    }
    left -= nb;
    kahan_add(Sa, Ca, pa.x + pa.y);
    kahan_add(Sb, Cb, pb.x + pb.y);
  }
}

// First D coordinates of a staged raw row (RAW floats, 16-byte aligned for RAW >= 4).
template <int D>
__device__ __forceinline__ void load_raw(const float* row, float* a) {
  constexpr int RAW = BaseShape<D>::RAW;
  if constexpr (RAW == 1) {
    a[0] = row[0];
  } else if constexpr (RAW == 2) {
    const float2 v = *reinterpret_cast<const float2*>(row);
    a[0] = v.x; a[1] = v.y;
  } else {
    const float4 v = *reinterpret_cast<const float4*>(row);
    a[0] = v.x; a[1] = v.y; a[2] = v.z;
    if constexpr (D >= 4) a[3] = v.w;
    if constexpr (D == 5) a[4] = row[4];
  }
}

// Two forms of the exponent x = c |q - r|^2, c = -log2(e)/(2h^2):
//  * direct: differences q - r, D packed add + D packed fma + 1 packed mul
//    per two interactions; rounding changes a term by at most (D+4) u x
//    relative (x in natural units from here on);
//  * expanded about the query node's center m, with q~ = q - m, r~ = r - m:
//    x = A_q + B_r + sum_k W_qk r~_k, A_q = c|q~|^2, W_q = -2c q~, B_r = c|r~|^2
//    staged with the reference; the sum runs over 2^(B_r + W_q . r~) with D
//    packed fma per two interactions and is scaled by 2^A_q once per query
//    and tile (B_r + W_q . r~ = x - A_q lies between x and |c| |q~|^2, so it
//    cannot overflow, and it underflows only where 2^x does).  Its error in
//    x, with the rounding of q~ and r~ taken as a perturbation of the points
//    (2u), is at most u ((D+4) (|q~| + |r~|)^2 + D |r~|^2) / 2h^2: A_q and
//    B_r each take D + 1 roundings and c one, W_q . r~ one per product and
//    one per step of the chain of D fused multiply-adds, and that chain
//    starts from B_r, so each of its steps may also round away up to u |B_r|
//    (hence the D |r~|^2).  A run uses it when that is at most E for the
//    query box and the farthest corner of every reference box, or when
//    (10 D + 32) u rho_Q^2 / 2h^2 <= E for the query box radius rho_Q alone:
//    with |r~| <= |q~| + |q - r| and (a + b)^2 <= 2a^2 + 2b^2 the error is
//    then at most E + (4 D + 8) u x per term.  Otherwise the direct form.
//    E is a quarter of the float allowance eps_fp, so a term stays within
//    eps_fp whenever 2^-21 + eps_fp / 4 + (4 D + 8) u x <= eps_fp.

constexpr int kQCap = 128;  // queries of a run staged at a time

template <int D>
__global__ void __launch_bounds__(kBaseWarps * 32, 20 / kBaseWarps)
    k_base(TreeView Q, TreeView R, const int* __restrict__ rsorted, const int* __restrict__ ksorted, int n,
           const float* __restrict__ c2v, const float* __restrict__ inv2h2_up, double* __restrict__ gacc,
           unsigned long long* __restrict__ exp_ctr, float exp_err) {
  using SH = BaseShape<D>;
  constexpr int TILE = SH::TILE, RAW = SH::RAW, NV = SH::NV, SV = SH::SV;
  constexpr int QV = (D + 1 + 3) / 4;  // float4 per staged query: W (or q) then A
  // one tile per warp: raw rows land at the start of their pair slot and
  // each pair is rewritten in place into the interleaved form
  __shared__ __align__(16) float4 sT[kBaseWarps][(TILE / 2) * SV];
  __shared__ __align__(16) float4 sQ[kBaseWarps][kQCap * QV];
  __shared__ float2 sAcc[kBaseWarps][kQCap];
  __shared__ int sOff[kBaseWarps][2][kEntryChunk + 1];
  __shared__ int sRb[kBaseWarps][2][kEntryChunk];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long i0 = ((long)blockIdx.x * kBaseWarps + wib) * kEntryChunk;
  if (i0 >= n) return;
  const int m = (int)min((long)kEntryChunk, n - i0);
  const unsigned FULL = 0xffffffffu;

  // ---- descriptors, one entry per lane
  int key = -1 - lane, rb = 0, rn = 0, qbeg = 0, qcnt = 0;
  float mc[D], rho2 = 0.f, far2 = 0.f, c2 = 0.f, i2h = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) mc[k] = 0.f;
  bool self = false;  // leave-one-out: the entry's nodes share points
  if (lane < m) {
    key = ksorted[i0 + lane];
    const int rv = rsorted[i0 + lane];
    const int r = rv & kNodeMask;
    self = ((rv >> kNodeBits) & kSelfFlag) != 0;
    const int hidx = key / Q.nn, q = key - hidx * Q.nn;
    rb = R.beg[r];
    rn = R.cnt[r];
    qbeg = Q.beg[q];
    qcnt = Q.cnt[q];
    c2 = c2v[hidx];
    i2h = inv2h2_up[hidx];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float lo = Q.lo[(size_t)q * D + k], hi = Q.hi[(size_t)q * D + k];
      mc[k] = 0.5f * (lo + hi);
      const float w = fmaxf(__fsub_ru(hi, mc[k]), __fsub_ru(mc[k], lo));
      rho2 = __fmaf_ru(w, w, rho2);
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float lo = R.lo[(size_t)r * D + k], hi = R.hi[(size_t)r * D + k];
      const float w = fmaxf(fabsf(__fsub_ru(hi, mc[k])), fabsf(__fsub_rd(lo, mc[k])));
      far2 = __fmaf_ru(w, w, far2);
    }
  }
  const int keyp = __shfl_up_sync(FULL, key, 1);
  const unsigned starts = __ballot_sync(FULL, lane < m && (lane == 0 || key != keyp));
  auto run_end = [&](int t) -> int {
    const unsigned later = starts & ~((2u << t) - 1u);
    return later ? __ffs(later) - 1 : m;
  };
  // offset table of run [t, e) in slot sl; returns the run's reference count
  auto build_table = [&](int t, int e, int sl) -> int {
    const int in_run = (lane >= t && lane < e) ? rn : 0;
    int incl = in_run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const int tot = __shfl_sync(FULL, incl, 31);
    if (lane >= t && lane < e) {
      sOff[wib][sl][lane - t] = incl - in_run;
      sRb[wib][sl][lane - t] = rb;
    }
    if (lane == 0) sOff[wib][sl][e - t] = tot;
    __syncwarp();
    return tot;
  };
  // raw rows [j0, j0 + tn) of the run in table slot sl (ne entries) -> sRaw, asynchronously
  auto issue = [&](int sl, int ne, int j0, int tn) {
    int u = -1;
    for (int j = lane; j < tn; j += 32) {
      const int J = j0 + j;
      if (u < 0) {
        int lo = 0, hi = ne;  // sOff[lo] <= J < sOff[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (sOff[wib][sl][mid] <= J) lo = mid; else hi = mid;
        }
        u = lo;
      } else {
        while (sOff[wib][sl][u + 1] <= J) ++u;
      }
      const float* src = R.pts + (size_t)(sRb[wib][sl][u] + J - sOff[wib][sl][u]) * RAW;
      float* dst = reinterpret_cast<float*>(&sT[wib][(j >> 1) * SV]) + (j & 1) * RAW;
      if constexpr (RAW * 4 <= 16) {
        cp_async_row(dst, src, RAW * 4);
      } else {
#pragma unroll
        for (int c = 0; c < RAW * 4 / 16; ++c) cp_async_row(dst + 4 * c, src + 4 * c, 16);
      }
    }
    cp_async_commit();
  };

  // current segment: run [t, e) (table slot ts), query block qs, tile j0
  int t = 0, e = run_end(0), ts = 0, qs = 0, j0 = 0;
  int tot = build_table(t, e, ts);
  // run parameters (warp-uniform), refreshed when the run changes
  float c2r = 0.f, m_[D];
  int qb = 0, qn = 0, hidx = 0;
  bool expanded = false, self_run = false;
  bool new_run = true;
  int g = 32, lgg = 5, ngrp = 1, ql = 0, gid = 0, qcnt_blk = 0;
  while (true) {
    if (new_run) {
      c2r = __shfl_sync(FULL, c2, t);
      qb = __shfl_sync(FULL, qbeg, t);
      qn = __shfl_sync(FULL, qcnt, t);
      hidx = __shfl_sync(FULL, key, t) / Q.nn;
#pragma unroll
      for (int k = 0; k < D; ++k) m_[k] = __shfl_sync(FULL, mc[k], t);
      const float rq2 = __shfl_sync(FULL, rho2, t);
      const float f2 = __uint_as_float(
          __reduce_max_sync(FULL, (lane >= t && lane < e) ? __float_as_uint(far2) : 0u));
      const float span = __fadd_ru(__fsqrt_ru(rq2), __fsqrt_ru(f2));
      const float uu = 5.9604645e-08f * __shfl_sync(FULL, i2h, t);
      // a run with a self entry takes the direct form, which leaves the
      // self interaction out exactly
      self_run = __any_sync(FULL, lane >= t && lane < e && self);
      expanded = !self_run && ((float)(D + 4) * uu * span * span + (float)D * uu * f2 <= exp_err ||
                               (float)(10 * D + 32) * uu * rq2 <= exp_err);
      if (expanded && lane == 0) atomicAdd(exp_ctr, (unsigned long long)qn * tot);
      new_run = false;
    }
    if (j0 == 0) {
      // a new query block: stage its queries (W and A, or the point) and clear its sums
      qcnt_blk = min(kQCap, qn - qs);
      g = pick_group(qcnt_blk, tot);
      lgg = 31 - __clz(g);
      ngrp = 32 >> lgg;
      ql = lane & (g - 1);
      gid = lane >> lgg;
      for (int qi = lane; qi < qcnt_blk; qi += 32) {
        float v[D];
        load_point<D>(Q.pts + (size_t)(qb + qs + qi) * Q.dp, v);
        float f[4 * QV];
#pragma unroll
        for (int i = 0; i < 4 * QV; ++i) f[i] = 0.f;
        float a2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float tq = v[k] - m_[k];
          a2 = fmaf(tq, tq, a2);
          f[k] = expanded ? -2.f * c2r * tq : v[k];
        }
        f[D] = c2r * a2;
#pragma unroll
        for (int i = 0; i < QV; ++i) sQ[wib][qi * QV + i] = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
        sAcc[wib][qi] = make_float2(0.f, 0.f);
      }
    }
    const int tn = min(TILE, tot - j0);
    // reference pairs, padded with zero-weight pairs to a multiple of the
    // lane groups so that every lane runs the same number of steps
    const int np2 = (((tn + 1) >> 1) + ngrp - 1) & ~(ngrp - 1);
    issue(ts, e - t, j0, tn);
    cp_async_wait_all();
    __syncwarp();
    // interleave: lane per reference pair
    for (int jp = lane; jp < np2; jp += 32) {
      const bool has_a = 2 * jp < tn, has_b = 2 * jp + 1 < tn;
      float a[D], b[D];
#pragma unroll
      for (int k = 0; k < D; ++k) a[k] = b[k] = 0.f;
      const float* slot = reinterpret_cast<const float*>(&sT[wib][jp * SV]);
      if (has_a) load_raw<D>(slot, a);
      if (has_b) load_raw<D>(slot + RAW, b);
      float f[4 * NV];
#pragma unroll
      for (int i = 0; i < 4 * NV; ++i) f[i] = 0.f;
      if (expanded) {
        float ba = 0.f, bb = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float ra = has_a ? a[k] - m_[k] : 0.f, rbv = has_b ? b[k] - m_[k] : 0.f;
          f[2 * k] = ra;
          f[2 * k + 1] = rbv;
          ba = fmaf(ra, ra, ba);
          bb = fmaf(rbv, rbv, bb);
        }
        f[2 * D] = has_a ? c2r * ba : -1.0e30f;
        f[2 * D + 1] = has_b ? c2r * bb : -1.0e30f;
      } else {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          f[2 * k] = has_a ? -a[k] : kFarNeg;
          f[2 * k + 1] = has_b ? -b[k] : kFarNeg;
        }
        if (self_run) {
          // the references' point indices, for the self test
          int ga = -1, gb = -1;
          for (int s2 = 0; s2 < 2; ++s2) {
            const int J = j0 + 2 * jp + s2;
            if (J >= j0 + tn) break;
            int lo = 0, hi = e - t;  // sOff[lo] <= J < sOff[hi]
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (sOff[wib][ts][mid] <= J) lo = mid; else hi = mid;
            }
            const int g = sRb[wib][ts][lo] + J - sOff[wib][ts][lo];
            if (s2 == 0) ga = g; else gb = g;
          }
          f[2 * D] = __int_as_float(ga);
          f[2 * D + 1] = __int_as_float(gb);
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v)
        sT[wib][jp * SV + v] = make_float4(f[4 * v], f[4 * v + 1], f[4 * v + 2], f[4 * v + 3]);
    }
    __syncwarp();
    // the next segment: next tile, else next query block, else next run
    int nt = t, ne = e, nts = ts, nqs = qs, nj0 = j0 + TILE, ntot = tot;
    const bool last_tile = nj0 >= tot;
    if (last_tile) {
      nj0 = 0;
      nqs = qs + kQCap;
      if (nqs >= qn) {
        nqs = 0;
        nt = e;
        if (nt < m) {
          ne = run_end(nt);
          nts = ts ^ 1;
          ntot = build_table(nt, ne, nts);
        }
      }
    }

    // sum this tile for every query of the block, into the block's sums
    const float2 c2p = make_float2(c2r, c2r);
    for (int q0 = 0; q0 < qcnt_blk; q0 += 2 * g) {
      const int qia = q0 + ql, qib = q0 + g + ql;
      const bool oka = qia < qcnt_blk, okb = qib < qcnt_blk;
      float2 wqa[D], wqb[D];
      {
        float fa[4 * QV], fb[4 * QV];
#pragma unroll
        for (int i = 0; i < QV; ++i) {
          const float4 va = sQ[wib][(oka ? qia : 0) * QV + i];
          const float4 vb = sQ[wib][(okb ? qib : 0) * QV + i];
          fa[4 * i] = va.x; fa[4 * i + 1] = va.y; fa[4 * i + 2] = va.z; fa[4 * i + 3] = va.w;
          fb[4 * i] = vb.x; fb[4 * i + 1] = vb.y; fb[4 * i + 2] = vb.z; fb[4 * i + 3] = vb.w;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
          wqa[k] = make_float2(fa[k], fa[k]);
          wqb[k] = make_float2(fb[k], fb[k]);
        }
      }
      float Sa = 0.f, Ca = 0.f, Sb = 0.f, Cb = 0.f;
      if (expanded)
        base_tile_sums<D, true>(sT[wib], np2, gid, ngrp, wqa, wqb, c2p, Sa, Ca, Sb, Cb);
      else if (self_run)
        base_tile_sums_loo<D>(sT[wib], np2, gid, ngrp, wqa, wqb, c2p, oka ? qb + qs + qia : -2,
                              okb ? qb + qs + qib : -2, Sa, Ca, Sb, Cb);
      else
        base_tile_sums<D, false>(sT[wib], np2, gid, ngrp, wqa, wqb, c2p, Sa, Ca, Sb, Cb);
      float va = Sa - Ca, vb = Sb - Cb;
      for (int o = g; o < 32; o <<= 1) {
        va += __shfl_xor_sync(FULL, va, o);
        vb += __shfl_xor_sync(FULL, vb, o);
      }
      if (gid == 0 && oka) {
        float2 acc = sAcc[wib][qia];
        kahan_add(acc.x, acc.y, va);
        sAcc[wib][qia] = acc;
      }
      if (gid == 0 && okb) {
        float2 acc = sAcc[wib][qib];
        kahan_add(acc.x, acc.y, vb);
        sAcc[wib][qib] = acc;
      }
    }
    if (last_tile) {
      // the block's sums, scaled by 2^A_q in the expanded form, one atomic per query
      __syncwarp();
      for (int qi = lane; qi < qcnt_blk; qi += 32) {
        const float2 acc = sAcc[wib][qi];
        float v = acc.x - acc.y;
        if (expanded) v *= exp2f(reinterpret_cast<const float*>(&sQ[wib][qi * QV])[D]);
        atomicAdd(&gacc[(size_t)hidx * Q.n + qb + qs + qi], (double)v);
      }
    }
    __syncwarp();
    if (nt >= m) break;
    if (nt != t) new_run = true;
    t = nt;
    e = ne;
    ts = nts;
    qs = nqs;
    j0 = nj0;
    tot = ntot;
  }
}

// D >= 6: exact sums in the direct form over the same sorted entries and
// runs as k_base, with the dimension padded to DM = 8, 16 or 32 (the
// tree's rows are zero-padded, so the extra coordinates add nothing).  A
// run's references are staged in shared memory a tile at a time, negated,
// as interleaved pairs (r_j, r_j+1 coordinate by coordinate, each pair slot
// padded by 16 bytes so that lane groups reading different pairs do not
// collide on banks); up to 128 of the run's queries are kept in flight,
// 32 per query block, a lane holding one query of a block and, for blocks
// of fewer than 32 queries, sharing the references with the other lanes of
// that query.  Per two interactions: DM packed subtractions and FMAs, one
// packed multiply, two ex2; blocks of 8 steps summed in float32 and added
// with Kahan compensation (so the rounding is that of the D <= 5 direct form,
// at most (D+4) u x per term).
constexpr int kHdQBlocks = 4;  // query blocks of 32 in flight per pass

// Reference pairs per tile, the largest that keeps the blocks per SM that
// the registers allow (4 at DM = 16, 2 at DM = 32): at DM = 32, 48 pairs ran
// the direct form 25% faster than 16 and 8% faster than 32 (64 would leave
// one block per SM); at DM = 16, 40 pairs 1.6% faster than 32, and 64 no
// faster than 40.
template <int DM>
struct HdShape {
  static constexpr int TP = DM == 8 ? 64 : DM == 16 ? 40 : 48;   // reference pairs per tile
  static constexpr int PS = 2 * DM + 4;                          // floats per pair slot
};

// Eight warps per block: one-warp blocks (more registers, no spills) ran
// the D = 16 direct form 6% slower.
constexpr int kHdWarps = 8;
// the block's reference tiles, in dynamic shared memory (past the 48 KB
// of a static allocation for the larger tiles)
template <int DM>
constexpr int hd_smem() { return kHdWarps * HdShape<DM>::TP * HdShape<DM>::PS * (int)sizeof(float); }
template <int DM>
__global__ void __launch_bounds__(kHdWarps * 32) k_base_hd(TreeView Q, TreeView R, const int* __restrict__ rsorted,
                                                const int* __restrict__ ksorted, int n,
                                                const float* __restrict__ c2v,
                                                const unsigned char* __restrict__ tcflag,
                                                double* __restrict__ gacc) {
  constexpr int TP = HdShape<DM>::TP, PS = HdShape<DM>::PS;
  extern __shared__ __align__(16) float sHd[];  // kHdWarps tiles of TP * PS floats
  __shared__ int sOff[kHdWarps][kEntryChunk + 1], sRb[kHdWarps][kEntryChunk];
  const unsigned FULL = 0xffffffffu;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long i0 = ((long)blockIdx.x * kHdWarps + wib) * kEntryChunk;
  if (i0 >= n) return;
  const int m = (int)min((long)kEntryChunk, n - i0);
  const int dpr = R.dp, dpq = Q.dp;
  int key = -1 - lane, rb = 0, rn = 0, qbeg = 0, qcnt = 0;
  bool self = false;  // leave-one-out: the entry's nodes share points
  if (lane < m) {
    key = ksorted[i0 + lane];
    const int rv = rsorted[i0 + lane];
    const int r = rv & kNodeMask;
    self = ((rv >> kNodeBits) & kSelfFlag) != 0;
    const int q = key % Q.nn;
    rb = R.beg[r];
    rn = R.cnt[r];
    qbeg = Q.beg[q];
    qcnt = Q.cnt[q];
  }
  const int keyp = __shfl_up_sync(FULL, key, 1);
  const unsigned starts = __ballot_sync(FULL, lane < m && (lane == 0 || key != keyp));
  float* T = sHd + (size_t)wib * TP * PS;
  int t = 0;
  while (t < m) {
    const unsigned later = starts & ~((2u << t) - 1u);
    const int e = later ? __ffs(later) - 1 : m;
    // the run's reference table
    const int in_run = (lane >= t && lane < e) ? rn : 0;
    int incl = in_run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const int tot = __shfl_sync(FULL, incl, 31);
    if (lane >= t && lane < e) {
      sOff[wib][lane - t] = incl - in_run;
      sRb[wib][lane - t] = rb;
    }
    if (lane == 0) sOff[wib][e - t] = tot;
    const int key_t = __shfl_sync(FULL, key, t);
    const int hidx = key_t / Q.nn;
    const int qb = __shfl_sync(FULL, qbeg, t), qn = __shfl_sync(FULL, qcnt, t);
    const float c2 = c2v[hidx];
    const float2 c2p = make_float2(c2, c2);
    const bool loo = __any_sync(FULL, lane >= t && lane < e && self);
    if (tcflag[i0 + t]) {
      // a run of the tensor form (k_tc_plan) is summed by k_base_tc
      __syncwarp();
      t = e;
      continue;
    }
    __syncwarp();
    for (int qs = 0; qs < qn; qs += 32 * kHdQBlocks) {
      const int nblk = min(kHdQBlocks, (qn - qs + 31) / 32);
      float S[kHdQBlocks], Cc[kHdQBlocks];
#pragma unroll
      for (int b = 0; b < kHdQBlocks; ++b) S[b] = Cc[b] = 0.f;
      for (int j0 = 0; j0 < tot; j0 += 2 * TP) {
        const int tn = min(2 * TP, tot - j0);
        const int np = (tn + 1) >> 1;
        // stage references j0 .. j0+tn-1 as interleaved pairs; a missing
        // partner gets far coordinates (its kernel value is 0)
        {
          int u = 0;
          for (int jj = lane; jj < 2 * np; jj += 32) {
            const int J = j0 + jj;
            float* slot = T + (jj >> 1) * PS + (jj & 1);
            if (J < tot) {
              while (sOff[wib][u + 1] <= J) ++u;
              const int g = sRb[wib][u] + J - sOff[wib][u];
              const float* src = R.pts + (size_t)g * dpr;
#pragma unroll
              for (int k = 0; k < DM; ++k) slot[2 * k] = k < dpr ? -src[k] : 0.f;
              slot[2 * DM] = __int_as_float(g);  // the point index, for the self test
            } else {
#pragma unroll
              for (int k = 0; k < DM; ++k) slot[2 * k] = -1.0e18f;
              slot[2 * DM] = __int_as_float(-1);
            }
          }
        }
        __syncwarp();
        for (int b = 0; b < nblk; ++b) {
          const int qbk = min(32, qn - qs - 32 * b);
          const int QL = qbk > 16 ? 32 : qbk > 8 ? 16 : qbk > 4 ? 8 : qbk > 2 ? 4 : qbk > 1 ? 2 : 1;
          const int NG = 32 / QL, ql = lane & (QL - 1), grp = lane / QL;
          const bool vq = ql < qbk;
          const int qi = qs + 32 * b + ql;
          const int qg = vq ? qb + qi : -2;  // the query's point index
          float2 qq[DM];
#pragma unroll
          for (int k = 0; k < DM; ++k) {
            const float v = (vq && k < dpq) ? Q.pts[(size_t)(qb + qi) * dpq + k] : 0.f;
            qq[k] = make_float2(v, v);
          }
          float2 blk = make_float2(0.f, 0.f);
          int steps = 0;
          for (int p = grp; p < np; p += NG) {
            const float4* rp = reinterpret_cast<const float4*>(T + p * PS);
            float2 d2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < DM; k += 2) {
              const float4 r4 = rp[k >> 1];  // -(r_j,k, r_j+1,k, r_j,k+1, r_j+1,k+1)
              const float2 da = __fadd2_rn(qq[k], make_float2(r4.x, r4.y));
              const float2 db = __fadd2_rn(qq[k + 1], make_float2(r4.z, r4.w));
              d2 = __ffma2_rn(da, da, d2);
              d2 = __ffma2_rn(db, db, d2);
            }
            const float2 x = __fmul2_rn(d2, c2p);
            float e0 = ex2_approx(x.x), e1 = ex2_approx(x.y);
            if (loo) {  // leave-one-out: a query meets its own index with weight 0
              const int2 ids = *reinterpret_cast<const int2*>(T + p * PS + 2 * DM);
              if (ids.x == qg) e0 = 0.f;
              if (ids.y == qg) e1 = 0.f;
            }
            blk = __fadd2_rn(blk, make_float2(e0, e1));
            if (++steps == 8) {
              steps = 0;
              kahan_add(S[b], Cc[b], blk.x + blk.y);
              blk = make_float2(0.f, 0.f);
            }
          }
          kahan_add(S[b], Cc[b], blk.x + blk.y);
        }
        __syncwarp();
      }
      // the lane groups of each query block hold parts of its sums
      for (int b = 0; b < nblk; ++b) {
        const int qbk = min(32, qn - qs - 32 * b);
        const int QL = qbk > 16 ? 32 : qbk > 8 ? 16 : qbk > 4 ? 8 : qbk > 2 ? 4 : qbk > 1 ? 2 : 1;
        float v = S[b] - Cc[b];
        for (int o = QL; o < 32; o <<= 1) v += __shfl_xor_sync(FULL, v, o);
        const int ql = lane & (QL - 1);
        if (lane < QL && ql < qbk) atomicAdd(&gacc[(size_t)hidx * Q.n + qb + qs + 32 * b + ql], (double)v);
      }
    }
    __syncwarp();
    t = e;
  }
}

template <int DM>
cudaError_t launch_base_hd(int g, const TreeView& Q, const TreeView& R, const int* rsorted, const int* ksorted,
                           int n, const float* c2, const unsigned char* tcflag, double* gacc, cudaStream_t s) {
  constexpr int smem = hd_smem<DM>();
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_base_hd<DM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  k_base_hd<DM><<<g, kHdWarps * 32, smem, s>>>(Q, R, rsorted, ksorted, n, c2, tcflag, gacc);
  return cudaGetLastError();
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
// sum over the multi-indices of M[alpha] prod_k H[j][k][alpha_k] for NQ
// points j, nested one dimension at a time (radix PM, dimension K upward,
// the last dimension contiguous in M): P + P/PM + ... fma per point.
template <int D, int PM, int K, int NQ>
__device__ __forceinline__ void eval_nested(const float* __restrict__ M, const float (*H)[D][PM], float* out) {
  constexpr int STRIDE = ipow_c(PM, D - 1 - K);
  float acc[NQ];
#pragma unroll
  for (int j = 0; j < NQ; ++j) acc[j] = 0.f;
#pragma unroll
  for (int e = 0; e < PM; ++e) {
    if constexpr (K == D - 1) {
      const float m = M[e];
#pragma unroll
      for (int j = 0; j < NQ; ++j) acc[j] = fmaf(H[j][K][e], m, acc[j]);
    } else {
      float in[NQ];
      eval_nested<D, PM, K + 1, NQ>(M + e * STRIDE, H, in);
#pragma unroll
      for (int j = 0; j < NQ; ++j) acc[j] = fmaf(H[j][K][e], in[j], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < NQ; ++j) out[j] = acc[j];
}

// Far-field value at NQ queries of this lane (q0 + lane + 32 j).
template <int D, int NQ>
__device__ __forceinline__ void farfield_points(const TreeView& Q, const float* Ms, const CenterHL* cR,
                                                float sf, int qb, int qn, int q0, int lane,
                                                double* __restrict__ gout, float sub) {
  constexpr int PM = pmax_of(D);
  float H[NQ][D][PM];
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    const int qi = q0 + lane + 32 * j;
    float v[D];
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = cR[k].hi;
    if (qi < qn) load_point<D>(Q.pts + (size_t)(qb + qi) * Q.dp, v);
#pragma unroll
    for (int k = 0; k < D; ++k) hermite_f32<PM>(minus_center(v[k], cR[k]) * sf, H[j][k]);
  }
  float acc[NQ];
  eval_nested<D, PM, 0, NQ>(Ms, H, acc);
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    const int qi = q0 + lane + 32 * j;
    if (qi < qn) atomicAdd(&gout[qb + qi], (double)(acc[j] - sub));
  }
}

// Four warps per block (one action each): warps of one block wait on the
// slowest of them; 1, 2, 4, 8 warps measured 0.52, 0.49, 0.49, 0.54 ms.
constexpr int kFarWarps = 4;
template <int D>
__global__ void __launch_bounds__(kFarWarps * 32) k_farfield(TreeView Q, TreeView R,
                                                 const Action* __restrict__ list, int n,
                                                 const float* __restrict__ sfv,
                                                 double* __restrict__ gacc) {
  constexpr int PM = pmax_of(D);
  constexpr int P = ipow_c(PM, D);
  __shared__ float sM[kFarWarps][P];
  const int wib = threadIdx.x >> 5;
  const int w = blockIdx.x * kFarWarps + wib;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const Action a = list[w];
  const float sf = sfv[a.h];
  float* Ms = sM[wib];
  // a summary over a node holding the query itself (leave-one-out sums)
  // loses its exact self term 1 (subtracted in float32: one more rounding
  // of the value, inside the factor 2 of its rounding allowance; a float64
  // subtraction per query kept the FP64 pipe at 46%)
  const float sub = (a.p & kSelfFlag) ? 1.f : 0.f;
  stage_moments<D, PM, P>(R.mnorm + (size_t)a.r * P, R.whalf[a.r] * sf, a.p & kOrderMask, Ms, lane);
  __syncwarp();
  CenterHL cR[D];
#pragma unroll
  for (int k = 0; k < D; ++k) cR[k] = center_hl(R, a.r, k);
  const int qb = Q.beg[a.q], qn = Q.cnt[a.q];
  // two queries per lane share every moment load while more than 32 remain
  double* gout = gacc + (size_t)a.h * Q.n;
  for (int q0 = 0; q0 < qn;) {
    if (qn - q0 > 32) {
      farfield_points<D, 2>(Q, Ms, cR, sf, qb, qn, q0, lane, gout, sub);
      q0 += 64;
    } else {
      farfield_points<D, 1>(Q, Ms, cR, sf, qb, qn, q0, lane, gout, sub);
      q0 += 32;
    }
  }
}

// ------------------------------------------------------------ direct local
// AccumulateDirectLocalMoment:
// L_beta(Q) += ((-1)^{|beta|}/beta!) sum_{r in R} h_beta((Q.c - r)/sqrt(2h^2)).
// The list is sorted by (bandwidth, query node) like the base case, and
// the warps split the sorted entries' references evenly (k_local below); a
// run of one query node is one concatenated list of references, taken in
// batches of 32 (one per lane, the next batch's point loaded while the
// current one is summed).  The coefficient sum_r prod_k h_{beta_k}(t_rk) factors over
// dimensions, so a lane owns the coefficients of one prefix (beta_0 ..
// beta_{D-B-1}) and all PM^B values of the last B digits: per reference it
// forms the prefix product once and multiplies it out over the block, with
// the 1-D Hermite rows tabulated in shared memory by the reference's lane.
// Lanes of one prefix split the batch into streams, reduced at the end of
// the run; each lane's batch sums are Kahan-compensated.  An entry of order
// p contributes only to beta < p: its rows are zero past p.
template <int D>
struct LocalShape {
  static constexpr int PM = pmax_of(D);
  static constexpr int P = ipow_c(PM, D);
  static constexpr int B = D <= 2 ? 1 : 2;             // block digits
  static constexpr int NB = ipow_c(PM, B);             // coefficients per lane
  static constexpr int NPRE = ipow_c(PM, D - B);       // prefixes
  static constexpr int NSTR = 32 / NPRE;               // streams per prefix
};

// Local moments over a balanced split: every sorted entry weighs its
// reference count plus kEntryCost (its share of the fixed per-entry and
// per-run work, in reference units), the weights form one sequence (entry e
// covers [eoff[e], eoff[e+1]): kEntryCost units of set-up, then one unit
// per reference), and warp k of NW takes the k-th of NW equal slices of it,
// so no warp waits on one large reference node.  A warp walks its slice 32
// entries at a time; consecutive entries of one (bandwidth, query node) key
// form a run whose coefficients accumulate in registers, and they are
// added to the node's moments (float64 atomics) when the key changes or the
// slice ends.  Each reference is tabulated once per lane (Hermite values
// h_e((Q.c - r) s), zero beyond the entry's order), and lane (stream,
// prefix) owns the coefficients of one prefix of the multi-index.
constexpr int kEntryCost = 8;  // measured: 4, 8, 16, 32, 64, 128 -> 0.69, 0.69, 0.70, 0.74, 0.82, 0.96 ms
template <int D>
__global__ void __launch_bounds__(kT, 3) k_local(TreeView Q, TreeView R, const int* __restrict__ rsorted,
                                                 const int* __restrict__ ksorted,
                                                 const long long* __restrict__ eoff, int n,
                                                 const float* __restrict__ sfv,
                                                 double* __restrict__ L, int* __restrict__ pused) {
  using LS = LocalShape<D>;
  constexpr int PM = LS::PM, P = LS::P, B = LS::B, NB = LS::NB, NPRE = LS::NPRE, NSTR = LS::NSTR;
  constexpr int NB2 = NB / 2;
  constexpr int S = (P + 31) / 32;
  constexpr int kFlush = 8;  // batches between compensated additions
  __shared__ __align__(16) float sH[kWarpsPerBlock][32][D][PM];
  __shared__ float sRed[kWarpsPerBlock][NSTR][P];
  __shared__ int sCum[kWarpsPerBlock][33], sRs[kWarpsPerBlock][32], sRp[kWarpsPerBlock][32];
  const unsigned FULL = 0xffffffffu;
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * kWarpsPerBlock + wib, NW = (long long)gridDim.x * kWarpsPerBlock;
  const long long T = eoff[n];
  const long long per = T / NW, extra = T % NW;
  const long long lo = per * gw + min(gw, extra);
  const long long hi = lo + per + (gw < extra ? 1 : 0);
  if (lo >= hi) return;
  // the entry holding reference lo: the last e with eoff[e] <= lo, found 32
  // probes at a time (eoff[base] <= lo holds throughout)
  int base = 0, len = n;
  while (len > 32) {
    const int step = (len + 31) / 32;
    const int idx = base + lane * step;
    const unsigned ok = __ballot_sync(FULL, idx < base + len && eoff[idx] <= lo);
    const int l = 31 - __clz(ok);
    const int nb = base + l * step;
    len = min(step, base + len - nb);
    base = nb;
  }
  int e = base + 31 - __clz(__ballot_sync(FULL, lane < len && eoff[base + lane] <= lo));

  // this lane's prefix, stream and prefix digits
  const int pre = lane % NPRE, str = lane / NPRE;
  int pd[D - B > 0 ? D - B : 1];
  {
    int v = pre;
#pragma unroll
    for (int k = D - B - 1; k >= 0; --k) { pd[k] = v % PM; v /= PM; }
  }
  float2 accS[NB2], accC[NB2], blk[NB2];
#pragma unroll
  for (int i = 0; i < NB2; ++i) accS[i] = accC[i] = blk[i] = make_float2(0.f, 0.f);
  int cur_key = -1, prun = 0, nb = 0;
  float sf = 0.f;
  CenterHL cQ[D];

  // adds the run's coefficients to the query node's moments and clears them
  auto flush = [&]() {
#pragma unroll
    for (int i = 0; i < NB2; ++i) {
      kahan_add(accS[i].x, accC[i].x, blk[i].x);
      kahan_add(accS[i].y, accC[i].y, blk[i].y);
      blk[i] = make_float2(0.f, 0.f);
    }
    nb = 0;
    if (str < NSTR) {
#pragma unroll
      for (int i = 0; i < NB2; ++i) {
        sRed[wib][str][pre * NB + 2 * i] = accS[i].x - accC[i].x;
        sRed[wib][str][pre * NB + 2 * i + 1] = accS[i].y - accC[i].y;
      }
    }
#pragma unroll
    for (int i = 0; i < NB2; ++i) accS[i] = accC[i] = make_float2(0.f, 0.f);
    __syncwarp();
    const int hidx = cur_key / Q.nn, q = cur_key - hidx * Q.nn;
    const size_t hq = (size_t)hidx * Q.nn + q;
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      const int idx = lane + 32 * sl;
      if (idx < P) {
        float cs = 0.f, cc = 0.f;
#pragma unroll
        for (int st = 0; st < NSTR; ++st) kahan_add(cs, cc, sRed[wib][st][idx]);
        const double v = (double)cs - (double)cc;
        if (v != 0.0) {
          int ab = 0;
          double f = 1.0;
          int w = idx;
#pragma unroll
          for (int k = D - 1; k >= 0; --k) { const int a = w % PM; w /= PM; ab += a; f *= fact_d(a); }
          atomicAdd(&L[hq * P + idx], ((ab & 1) ? -v : v) / f);
        }
      }
    }
    if (lane == 0) atomicMax(&pused[hq], prun);
    __syncwarp();
  };

  long long pos = lo;
  while (pos < hi) {
    // a window of 32 entries: the part of each entry's references inside
    // the slice (first point, count), orders, keys, and the window-wide
    // prefix of the counts
    const int ei = e + lane;
    int key = -1, rp = 0, rs = 0, c = 0;
    long long ee = T;
    if (ei < n) {
      key = ksorted[ei];
      const int v = rsorted[ei];
      rp = (v >> kNodeBits) & kOrderMask;
      const int rb = R.beg[v & kNodeMask];
      const long long eo = eoff[ei] + kEntryCost;
      ee = eoff[ei + 1];
      const long long s0 = max(pos, eo), s1 = min(hi, ee);
      if (s1 > s0) {
        c = (int)(s1 - s0);
        rs = rb + (int)(s0 - eo);
        // a node holding the query itself (leave-one-out sums): the slice
        // with the entry's first reference takes the self term 1 off L_0
        if (((v >> kNodeBits) & kSelfFlag) && s0 == eo) atomicAdd(&L[(size_t)key * P], -1.0);
      }
    }
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    sCum[wib][lane] = incl - c;
    sRs[wib][lane] = rs;
    sRp[wib][lane] = rp;
    if (lane == 31) sCum[wib][32] = incl;
    const long long wend = __shfl_sync(FULL, ee, 31);
    const int keyp = __shfl_up_sync(FULL, key, 1);
    const unsigned starts = __ballot_sync(FULL, lane == 0 || key != keyp);
    __syncwarp();
    int t = 0;
    while (t < 32) {
      const unsigned later = starts & ~((2u << t) - 1u);
      const int u = later ? __ffs(later) - 1 : 32;
      const int a = sCum[wib][t], b = sCum[wib][u];
      const int key_t = __shfl_sync(FULL, key, t);
      const int prun_t = __reduce_max_sync(FULL, (lane >= t && lane < u && c > 0) ? rp : 0);
      if (a < b && key_t >= 0) {
        if (key_t != cur_key) {
          if (cur_key >= 0) flush();
          cur_key = key_t;
          prun = 0;
          const int hidx = key_t / Q.nn, q = key_t - hidx * Q.nn;
          sf = sfv[hidx];
#pragma unroll
          for (int k = 0; k < D; ++k) cQ[k] = center_hl(Q, q, k);
        }
        prun = max(prun, prun_t);
        // references a .. b-1 of the window's concatenation, 32 per batch;
        // a lane's table cursor only moves forward
        int cur = t;
        auto fetch = [&](int J, float* pv, int& pp) {
          if (J < b) {
            while (cur + 1 < u && sCum[wib][cur + 1] <= J) ++cur;
            pp = sRp[wib][cur];
            load_point<D>(R.pts + (size_t)(sRs[wib][cur] + (J - sCum[wib][cur])) * R.dp, pv);
          } else {
            pp = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) pv[k] = 0.f;
          }
        };
        float pv[D];
        int pp = 0;
        fetch(a + lane, pv, pp);
        for (int j0 = a; j0 < b; j0 += 32) {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            float H[PM];
            hermite_f32<PM>(-minus_center(pv[k], cQ[k]) * sf, H);
#pragma unroll
            for (int e2 = 0; e2 < PM; e2 += 2)
              *reinterpret_cast<float2*>(&sH[wib][lane][k][e2]) =
                  make_float2(e2 < pp ? H[e2] : 0.f, e2 + 1 < pp ? H[e2 + 1] : 0.f);
          }
          __syncwarp();
          float nv[D];
          int np = 0;
          if (j0 + 32 < b) fetch(j0 + 32 + lane, nv, np);
          if (str < NSTR) {
            for (int j = str; j < 32; j += NSTR) {
              float pr = 1.f;
#pragma unroll
              for (int k = 0; k < D - B; ++k) pr *= sH[wib][j][k][pd[k]];
              const float2* hl = reinterpret_cast<const float2*>(&sH[wib][j][D - 1][0]);
              if constexpr (B == 1) {
                const float2 p2 = make_float2(pr, pr);
#pragma unroll
                for (int i = 0; i < NB2; ++i) blk[i] = __ffma2_rn(p2, hl[i], blk[i]);
              } else {
#pragma unroll
                for (int e1 = 0; e1 < PM; ++e1) {
                  const float t1 = pr * sH[wib][j][D - 2][e1];
                  const float2 t2 = make_float2(t1, t1);
#pragma unroll
                  for (int i = 0; i < PM / 2; ++i)
                    blk[e1 * (PM / 2) + i] = __ffma2_rn(t2, hl[i], blk[e1 * (PM / 2) + i]);
                }
              }
            }
          }
          if (++nb == kFlush) {
            nb = 0;
#pragma unroll
            for (int i = 0; i < NB2; ++i) {
              kahan_add(accS[i].x, accC[i].x, blk[i].x);
              kahan_add(accS[i].y, accC[i].y, blk[i].y);
              blk[i] = make_float2(0.f, 0.f);
            }
          }
          __syncwarp();
          if (j0 + 32 < b) {
#pragma unroll
            for (int k = 0; k < D; ++k) pv[k] = nv[k];
            pp = np;
          }
        }
      }
      t = u;
    }
    pos = max(pos, wend);
    e += 32;
    __syncwarp();
  }
  if (cur_key >= 0) flush();
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
  const int ord = a.p & kOrderMask;
  stage_moments<D, PM, P>(R.mnorm + (size_t)a.r * P, R.whalf[a.r] * (float)s, ord, sM[wib], lane);
  __syncwarp();
  const size_t hq = (size_t)a.h * Q.nn + a.q;
  if (lane == 0 && (a.p & kSelfFlag)) atomicAdd(&L[hq * P], -1.0);  // the node holds the query itself
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
      for (int k = D - 1; k >= 0; --k) { be[k] = v % PM; v /= PM; ab += be[k]; ok = ok && be[k] < ord; f *= fact_d(be[k]); }
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
  if (lane == 0) atomicMax(&pused[hq], ord);
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
    atomicAdd(&gacc[(size_t)a.h * Q.n + qb + qi],
              (double)(m0 * ex2_approx(d2 * c2)) - ((a.p & kSelfFlag) ? 1.0 : 0.0));
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
    atomicAdd(&L[hq], v - ((a.p & kSelfFlag) ? 1.0 : 0.0));
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
  atomicAdd(&L[hq], R.mom[a.r] * exp(-d2 / (2.0 * h * h)) - ((a.p & kSelfFlag) ? 1.0 : 0.0));
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
  if (Q.d <= 5) {
    const long warps = (n + kEntryChunk - 1) / kEntryChunk;
    const int g = (int)((warps + kBaseWarps - 1) / kBaseWarps);
    DISPATCH_D(Q.d, k_base<DD><<<g, kBaseWarps * 32, 0, s>>>(Q, R, rsorted, ksorted, n, b.c2, b.inv2h2_up,
                                                              b.gacc, b.base_exp, b.exp_err));
  } else {
    // which runs take the tensor form, then the direct-form runs (SIMT), then
    // the tensor-form runs
    const unsigned char* tcflag = nullptr;
    // after the scatter, off[key] is the end of the key's entries
    if ((e = launch_tc_plan(Q, R, b, rsorted, sc.cnt->as<int>(), sc.off->as<int>(), b.nh * Q.nn, n, *sc.plan,
                            &tcflag, s, launches)) != cudaSuccess)
      return e;
    const long warps = (n + kEntryChunk - 1) / kEntryChunk;
    const int g = (int)((warps + kHdWarps - 1) / kHdWarps);
    if (Q.dp <= 8)
      e = launch_base_hd<8>(g, Q, R, rsorted, ksorted, n, b.c2, tcflag, b.gacc, s);
    else if (Q.dp <= 16)
      e = launch_base_hd<16>(g, Q, R, rsorted, ksorted, n, b.c2, tcflag, b.gacc, s);
    else
      e = launch_base_hd<32>(g, Q, R, rsorted, ksorted, n, b.c2, tcflag, b.gacc, s);
    if (e != cudaSuccess) return e;
    ++*launches;
    if (sc.tc0 && (e = cudaEventRecord(sc.tc0, s)) != cudaSuccess) return e;
    if ((e = launch_tc_sums(Q, R, b, rsorted, n, *sc.plan, s, launches)) != cudaSuccess) return e;
    if (sc.tc1 && (e = cudaEventRecord(sc.tc1, s)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_farfield(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                            const Action* list, int n, BaseScratch&, cudaStream_t s, long long* launches) {
  if (n <= 0) return cudaSuccess;
  const int g = warp_grid(n);
  if (Q.d <= 5) {
    DISPATCH_D(Q.d, k_farfield<DD><<<(n + kFarWarps - 1) / kFarWarps, kFarWarps * 32, 0, s>>>(Q, R, list, n, b.sf,
                                                                                             b.gacc));
  } else {
    k_farfield_g<<<g, kT, 0, s>>>(Q, R, list, n, b.h, b.gacc);
  }
  ++*launches;
  return cudaGetLastError();
}

__global__ void k_entry_refs(const TreeView R, const int* __restrict__ rsorted, int n, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = R.cnt[rsorted[i] & kNodeMask] + kEntryCost;
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
    // reference counts of the sorted entries and their 64-bit prefix
    if ((e = sc.cnt->ensure((size_t)n * sizeof(int))) != cudaSuccess) return e;
    if ((e = sc.off->ensure(((size_t)n + 1) * sizeof(long long))) != cudaSuccess) return e;
    k_entry_refs<<<(n + kT - 1) / kT, kT, 0, s>>>(R, vsorted, n, sc.cnt->as<int>());
    ++*launches;
    if ((e = scan_exclusive64(sc.cnt->as<int>(), sc.off->as<long long>(), n, *sc.scan_tmp, s, launches)) !=
        cudaSuccess)
      return e;
    const int g = 3 * std::max(1, b.sms);  // every warp resident: three blocks per SM
    DISPATCH_D(Q.d, k_local<DD><<<g, kT, 0, s>>>(Q, R, vsorted, ksorted, sc.off->as<long long>(), n, b.sf, b.L,
                                                  b.pused));
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
