// common.cuh -- types and device helpers shared by the DFGT CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dfgt {

constexpr int kMaxD = 32;
constexpr int kWarp = 32;
constexpr int kMaxLeaf = 256;
typedef unsigned long long u64;

// Per-dimension expansion order limit p_max (Section 3.6, query-tree
// initialisation): 6 for D=2, 4 for D=3, 2 for D=4,5, 1 for D>=6.  D=1 is
// not listed in the paper; 8 is used.
__host__ __device__ constexpr int pmax_of(int D) {
  return D <= 1 ? 8 : D == 2 ? 6 : D == 3 ? 4 : D <= 5 ? 2 : 1;
}
__host__ __device__ constexpr int ipow_c(int b, int e) { return e <= 0 ? 1 : b * ipow_c(b, e - 1); }

// Row stride of the permuted point copy: float2 rows for D<=2, float4-aligned otherwise.
inline int padded_dim(int d) { return d <= 2 ? d : ((d + 3) & ~3); }

// Read-only view of a tree passed to kernels by value.
struct TreeView {
  const float* pts;    // [n][dp] points in leaf-contiguous (permuted) order
  const int* perm;     // [n] original index of each permuted point
  const float* lo;     // [nn][d] tight bounding box (Algorithm 2)
  const float* hi;     // [nn][d]
  const int* beg;      // [nn] first point of the node
  const int* cnt;      // [nn] number of points
  const int* left;     // [nn] first child, -1 for a leaf (second child = left+1)
  const int* parent;   // [nn] parent node, -1 for the root
  const double* mom;   // [nn][P] raw moments sum (r-c)^alpha/alpha! about the box center
  const float* chi;    // [nn][d] box center as a float pair chi + clo
  const float* clo;
  const float* whalf;  // [nn] largest half side w of the box (1 for a point)
  const float* mnorm;  // [nn][P] normalised moments m_alpha / w^|alpha| (|m~| <= |R|)
  const float* rad;    // [nn] radius of the node's points about its float box centre 0.5f (lo + hi), rounded up
  int n, d, dp, nn, pm, P;
};

// ---------------------------------------------------------------- math
// 2^x on the special-function unit (PTX ex2.approx, flush-to-zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr double kLog2e = 1.4426950408889634073599246810018921;

// Estimates below this go through the log-space pass of dfgt_sum_log: above
// it the dual-tree pass's float32 exact sums and its fixed-point lower
// bounds resolve the sum with room to spare (they need G >= ~1e-30).
constexpr double kLogFlag = 1e-20;

__host__ __device__ inline double fact_d(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

__device__ __forceinline__ double pow_int(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// Order-p truncation bound shared by far-field evaluation (Eq.
// error_bound_far_field) and direct local accumulation (Eq.
// error_bound_local): |R|/(1-r)^D sum_{k<D} C(D,k)(1-r^p)^k (r^p/sqrt(p!))^{D-k}.
__device__ inline double bound_farfield(double nR, int D, double r, int p) {
  const double rp = pow_int(r, p);
  const double a = 1.0 - rp;
  const double b = rp / sqrt(fact_d(p));
  double sum = 0.0, ak = 1.0, c = 1.0;  // c = C(D,k)
  for (int k = 0; k < D; ++k) {
    sum += c * ak * pow_int(b, D - k);
    ak *= a;
    c = c * (double)(D - k) / (double)(k + 1);
  }
  return nR * sum / pow_int(1.0 - r, D);
}

// Eq. error_bound_far_to_local with r < 1/2:
// |R|/(1-2r)^{2D} sum_{k<D} C(D,k) ((1-(2r)^p)^2)^k ((2r)^p(2-(2r)^p)/sqrt(p!))^{D-k}.
__device__ inline double bound_f2l(double nR, int D, double r, int p) {
  const double q = pow_int(2.0 * r, p);
  const double a = (1.0 - q) * (1.0 - q);
  const double b = q * (2.0 - q) / sqrt(fact_d(p));
  double sum = 0.0, ak = 1.0, c = 1.0;
  for (int k = 0; k < D; ++k) {
    sum += c * ak * pow_int(b, D - k);
    ak *= a;
    c = c * (double)(D - k) / (double)(k + 1);
  }
  return nR * sum / pow_int(1.0 - 2.0 * r, 2 * D);
}

// Rounding allowance for an order-p expansion evaluated in float32.  Each
// term of the truncated series is bounded (Szasz's inequality, as in the
// proofs of the truncation lemmas) so that the sum of absolute terms is at
// most |R| * S with S = ((1-r^p)/(1-r))^D (far field, local) or
// ((1-(2r)^p)/(1-2r))^{2D} (far to local); float32 evaluation, the shift
// of a local expansion to the leaf center, the float32 read-out and the
// coefficient conversions add at most c * u * |R| * S with u = 2^-24 and
// c = 2 (2 p^D + 6 p D + 6D + 16).
__host__ __device__ inline float fp_allowance_c(int p, int D) {
  float pD = 1.f;
  for (int i = 0; i < D; ++i) pD *= (float)p;
  return 2.f * (2.f * pD + 6.f * p * D + 6.f * D + 16.f);
}

// Float32 evaluations of the same bounds for order selection.  Every
// quantity is a sum or product of positive terms, so float32 evaluation is
// within ~16 ulps of the exact value; callers compare bound * (1 + 1e-4)
// against tau, which keeps every accepted order valid.
__device__ __forceinline__ float pow_int_f(float x, int e) {
  float r = 1.f;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

__device__ __forceinline__ float rsqrt_fact_f(int p) {
  // 1/sqrt(p!) for p = 0..8, as a chain of selects (no indexed local array)
  float t = 1.f;
  t = p == 2 ? 0.70710678f : t;
  t = p == 3 ? 0.40824829f : t;
  t = p == 4 ? 0.20412415f : t;
  t = p == 5 ? 0.091287093f : t;
  t = p == 6 ? 0.037267800f : t;
  t = p == 7 ? 0.014085904f : t;
  t = p >= 8 ? 0.0049801192f : t;
  return t;
}

// Eq. error_bound_far_field (and error_bound_local) plus the rounding
// allowance, float32; r < 1.
__device__ inline float bound_ff_total(float nR, int D, float r, int p) {
  const float rp = pow_int_f(r, p);
  const float a = 1.f - rp, b = rp * rsqrt_fact_f(p);
  float sum = 0.f, ak = 1.f, c = 1.f;
  for (int k = 0; k < D; ++k) {
    sum += c * ak * pow_int_f(b, D - k);
    ak *= a;
    c = c * (float)(D - k) / (float)(k + 1);
  }
  const float g = __frcp_rn(1.f - r);  // correctly rounded, as 1 / (1 - r)
  const float gD = pow_int_f(g, D);
  const float S = pow_int_f(a * g, D);
  const float cfp = fp_allowance_c(p, D) * 5.9604645e-08f;
  return nR * (sum * gD + cfp * S);
}

// Eq. error_bound_far_to_local plus the rounding allowance, float32; r < 1/2.
__device__ inline float bound_f2l_total(float nR, int D, float r, int p) {
  const float q = pow_int_f(2.f * r, p);
  const float a = (1.f - q) * (1.f - q), b = q * (2.f - q) * rsqrt_fact_f(p);
  float sum = 0.f, ak = 1.f, c = 1.f;
  for (int k = 0; k < D; ++k) {
    sum += c * ak * pow_int_f(b, D - k);
    ak *= a;
    c = c * (float)(D - k) / (float)(k + 1);
  }
  const float g = __frcp_rn(1.f - 2.f * r);  // correctly rounded, as 1 / (1 - 2r)
  const float g2D = pow_int_f(g, 2 * D);
  const float S = pow_int_f((1.f - q) * g, 2 * D);
  const float cfp = fp_allowance_c(p, D) * 5.9604645e-08f;
  return nR * (sum * g2D + cfp * S);
}

// ------------------------------------------------------------- atomics
__device__ __forceinline__ void atomic_min_f(float* a, float v) {
  if (v >= 0.f)
    atomicMin(reinterpret_cast<int*>(a), __float_as_int(v));
  else
    atomicMax(reinterpret_cast<unsigned*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float* a, float v) {
  if (v >= 0.f)
    atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned*>(a), __float_as_uint(v));
}

// Squared distance bounds of two boxes, Eqs. (6)-(7), and their largest
// sides, in float32 with directed rounding: dl2 never exceeds and du2 never
// falls below the exact value, and the sides are rounded up, so every
// kernel value and every truncation bound derived from them stays on the
// safe side.  (x + |x|)/2 summed over the two orderings of Eq. (6) is
// max(rl - qu, ql - ru, 0).
// For D >= 6 (the generic D = 0 instance with d >= 6) the bounds are
// tightened by the nodes' balls about their box centres c (radius r of the
// points, Q.rad / R.rad): every pair of points is at least |c_Q - c_R| -
// r_Q - r_R and at most |c_Q - c_R| + r_Q + r_R apart.  In many dimensions
// a kd box is much wider than the points it holds, and the box bound alone
// separates almost no pair; any valid pair of bounds serves the traversal
// (Theorem 3.3 needs only that the distances lie between them).
template <int D>
__device__ __forceinline__ void box_geometry(const TreeView& Q, int q, const TreeView& R, int r,
                                             float& dl2, float& du2, float& sideQ, float& sideR) {
  const int d = D > 0 ? D : Q.d;
  const bool ball = D == 0 && d >= 6;
  float c2dn = 0.f, c2up = 0.f;
  dl2 = du2 = sideQ = sideR = 0.f;
  for (int k = 0; k < d; ++k) {
    const float ql = Q.lo[(size_t)q * d + k], qu = Q.hi[(size_t)q * d + k];
    const float rl = R.lo[(size_t)r * d + k], ru = R.hi[(size_t)r * d + k];
    const float gap = fmaxf(0.f, fmaxf(__fsub_rd(rl, qu), __fsub_rd(ql, ru)));
    dl2 = __fmaf_rd(gap, gap, dl2);
    const float far = fmaxf(__fsub_ru(ru, ql), __fsub_ru(qu, rl));
    du2 = __fmaf_ru(far, far, du2);
    sideQ = fmaxf(sideQ, __fsub_ru(qu, ql));
    sideR = fmaxf(sideR, __fsub_ru(ru, rl));
    if (ball) {
      const float cq = 0.5f * (ql + qu), cr = 0.5f * (rl + ru);
      const float dn = cq >= cr ? __fsub_rd(cq, cr) : __fsub_rd(cr, cq);
      const float up = cq >= cr ? __fsub_ru(cq, cr) : __fsub_ru(cr, cq);
      c2dn = __fmaf_rd(dn, dn, c2dn);
      c2up = __fmaf_ru(up, up, c2up);
    }
  }
  if (ball) {
    const float rr = __fadd_ru(Q.rad[q], R.rad[r]);
    const float lo = __fsub_rd(__fsqrt_rd(c2dn), rr);
    if (lo > 0.f) dl2 = fmaxf(dl2, __fmul_rd(lo, lo));
    const float hi = __fadd_ru(__fsqrt_ru(c2up), rr);
    du2 = fminf(du2, __fmul_ru(hi, hi));
  }
}

// Bounds on the kernel over a node pair: Kl >= K(d^l) and Ku <= K(d^u).
// expf is within 2 ulps; the 1e-6 factors cover it.  Below the float32
// range (K < ~1e-38, exactly 0 past ~1e-45) Kl is not an upper bound, so a
// pair whose kernel underflows counts as contributing 0.  Every query's
// sum has at most N < 2^29 such terms, each below 1.2e-38, so for sums
// G >= 1e-30 (the range the exact float32 leaf sums need anyway) the
// change is below 7e-7 G, inside the float32 allowance of eps.
__device__ __forceinline__ float kernel_upper(float dl2, float inv2h2_dn) {
  return __fmul_ru(expf(-__fmul_rd(dl2, inv2h2_dn)), 1.000001f);
}
__device__ __forceinline__ float kernel_lower(float du2, float inv2h2_up) {
  return __fmul_rd(expf(-__fmul_ru(du2, inv2h2_up)), 0.999999f);
}

// Packed work item of the traversal: query node, reference node,
// bandwidth index and flags (bit 0: q was just split from its parent).
struct Pair {
  int q, r, h, flags;
};
// Summary action item: node pair, bandwidth index and expansion order.
struct Action {
  int q, r, h, p;
};

enum : int { kFlagSplitQ = 1 };
// Leave-one-out sums: an action or base entry whose reference node holds the
// query itself (the self term is removed exactly); kept above the order bits.
enum : int { kSelfFlag = 16, kOrderMask = 15 };

// Do the point ranges of node q of Q and node r of R (the same tree) meet?
__device__ __forceinline__ bool ranges_meet(const TreeView& Q, int q, const TreeView& R, int r) {
  const int qb = Q.beg[q], rb = R.beg[r];
  return qb < rb + R.cnt[r] && rb < qb + Q.cnt[q];
}
// Does node r of R hold every point of node q of Q (the same tree)?
__device__ __forceinline__ bool range_holds(const TreeView& R, int r, const TreeView& Q, int q) {
  const int qb = Q.beg[q], rb = R.beg[r];
  return rb <= qb && qb + Q.cnt[q] <= rb + R.cnt[r];
}

// Device status word bits (read back once per call).
enum : int {
  kStNonFinite = 1,   // a coordinate was NaN/Inf
  kStOverflow = 2,    // a work list ran out of room (retry with more)
  kStTimeout = 4,     // a bounded grid-barrier wait gave up
};

// ------------------------------------------------------- grid barrier
constexpr long long kSpinLimit = 1LL << 25;  // barrier polls before giving up (~1 s)

// How the grid barriers of one cooperative launch wait.  `limit` is the
// number of polls before a wait gives up.  `extra` > 0 makes every barrier
// wait for that many arrivals more than the grid has: no block can pass,
// so each one gives up at the first barrier, sets kStTimeout and returns
// (the error path of a wait that runs out, injected from the host).
struct BarrierCfg {
  long long limit = kSpinLimit;
  unsigned extra = 0;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch on a monotone arrival counter:
// every block passes the same sequence of barriers, so the k-th barrier
// opens when the counter reaches k * gridDim.x (`target`, kept by each
// block).  The wait is bounded: a block that polls cfg.limit times sets
// kStTimeout and leaves; every block returns false from then on, as it does
// once a non-finite coordinate has been seen.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* status, unsigned& target,
                                             const BarrierCfg& cfg) {
  __shared__ int s_ok;
  __syncthreads();
  target += gridDim.x + cfg.extra;
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    long long it = 0;
    while ((int)(ld_acquire(bar) - target) < 0) {
      if (++it > cfg.limit) {
        atomicOr(status, kStTimeout);
        break;
      }
    }
    __threadfence();
    s_ok = (*reinterpret_cast<volatile int*>(status) & (kStTimeout | kStNonFinite)) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace dfgt
