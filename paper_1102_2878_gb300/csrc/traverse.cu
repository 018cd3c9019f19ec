// traverse.cu -- level-synchronous dual-tree traversal (the DFGT recursion of
// Section 3.6, one round per sweep over a frontier of node pairs; all rounds
// run in one cooperative launch, phases separated by grid barriers).
//
// Every round classifies all frontier pairs (Q, R, h) at once:
//   * the distance-bound prune (the finite-difference approximation of the
//     predecessor dual-tree method, used in the proof of Theorem 3.3):
//     every query of Q gets |R|(K(d^l)+K(d^u))/2, error at most
//     |R|(K(d^l)-K(d^u))/2;
//   * otherwise ChooseBestMethod with FarFieldOrder, LocalAccumulationOrder
//     and ConvertFarFieldToLocalOrder picks far-field evaluation (F), direct
//     local accumulation (D) or far-to-local translation (T);
//   * otherwise a leaf-leaf pair goes to the exact base case (DFGTBase) and
//     any other pair is split into its child pairs for the next round.
// Both approximations are accepted only if their error is at most
// tau = eps |R| G^l(Q) / |R_total| (CanSummarize).  Summaries are only
// listed here; the action kernels run once over the complete lists after
// the traversal, since no decision depends on their results.
//
// Lower bound G^l(Q).  In a breadth-first order the exact base-case sums
// of the depth-first recursion are not yet known when a pair is decided,
// so G^l(Q) is built from the bounds delta^l = |R| K(d^u) of a partition
// of the reference set: every pair already decided for Q or an ancestor of
// Q, plus every pair of Q pending in this round.  Each such set of pairs
// covers every reference point exactly once (Theorem 3.2), and each
// delta^l is at most the true contribution of its reference node to any
// query of Q, so the sum is a valid lower bound -- all that Theorem 3.3
// needs.  Sums are kept in 64-bit fixed point (units of |R_total| 2^-62,
// rounded down), so they are exact, order-independent and deterministic.
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kT = 256;
constexpr float kMaxSummaryPoints = 4096.f;
constexpr int kSplitROnly = 1, kSplitQOnly = 2;

// Truncation of a non-negative float below 2^64 to an integer, by shifting
// its significand (integer instructions only).
__device__ __forceinline__ u64 f2u64_rz(float x) {
  const unsigned bits = __float_as_uint(x);
  const int e = (int)(bits >> 23) - 127;  // x = 1.m 2^e
  if (e < 0) return 0;
  const u64 m = (u64)((bits & 0x7fffffu) | 0x800000u);
  return e >= 23 ? m << (e - 23) : m >> (23 - e);
}

// A u64 as a float, rounded down.
__device__ __forceinline__ float u64_to_f_rd(u64 v) {
  return __fmaf_rd(__uint2float_rd((unsigned)(v >> 32)), 4294967296.f, __uint2float_rd((unsigned)v));
}

// Fixed-point units of a lower bound (rounded down).
__device__ __forceinline__ u64 to_fix_f(float nR, float K, float scale_dn) {
  return f2u64_rz(__fmul_rd(__fmul_rd(nR, K), scale_dn));
}

// FarFieldOrder / LocalAccumulationOrder: least p <= plim whose truncation
// bound plus float32 rounding allowance is <= tau; 0 = none (r >= 1).  The
// bound decreases with p, so the largest order is tried first and most
// pairs are rejected after one evaluation.
constexpr float kSafe = 1.0001f;  // covers float32 evaluation of the bounds

// r, |R| arrive rounded up and tau rounded down; every bound grows with r and |R|.
__device__ int order_ff(float r, float nR, int D, float tau, int plim) {
  if (!(r < 1.f)) return 0;
  if (bound_ff_total(nR, D, r, plim) * kSafe > tau) return 0;
  for (int p = 1; p < plim; ++p)
    if (bound_ff_total(nR, D, r, p) * kSafe <= tau) return p;
  return plim;
}

// ConvertFarFieldToLocalOrder; 0 = none (r >= 1/2).
__device__ int order_t(float r, float nR, int D, float tau, int plim) {
  if (!(r < 0.5f)) return 0;
  if (bound_f2l_total(nR, D, r, plim) * kSafe > tau) return 0;
  for (int p = 1; p < plim; ++p)
    if (bound_f2l_total(nR, D, r, p) * kSafe <= tau) return p;
  return plim;
}

// b^e for small non-negative integers (b^e < 2^64)
__device__ __forceinline__ unsigned long long ipow_u(int b, int e) {
  unsigned long long r = 1;
  for (int i = 0; i < e; ++i) r *= (unsigned long long)b;
  return r;
}

// Block-wide sum added with one atomic (every thread of the block calls it;
// scratch holds one word per warp).
__device__ __forceinline__ void warp_add_u64_block(unsigned long long* counter, unsigned long long v,
                                                   u64* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += scratch[w];
    if (t) atomicAdd(counter, t);
  }
}

// Round start: fold the previous round's decided bounds into `decided` and
// clear the per-round sums.
__device__ __forceinline__ void fold_phase(const TravBuffers& b, int total) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    b.decided[i] = __ldcg(b.decided + i) + __ldcg(b.incr + i);
    b.incr[i] = 0;
    b.lbsum[i] = 0;
  }
}

__global__ void k_init_frontier(Pair* F, int nh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nh) F[i] = Pair{0, 0, i, 0};
}

__device__ __forceinline__ Pair load_pair(const Pair* F, int i) {
  const int4 v = __ldcg(reinterpret_cast<const int4*>(F) + i);
  return Pair{v.x, v.y, v.z, v.w};
}

// Pending lower bounds: inherit the decided bound of a just-split parent,
// then add delta^l of every pending pair of the node.  Pair i is handled by
// the same thread as in the classification that follows.
template <int D>
__device__ __forceinline__ void lb_phase(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                                         const Pair* __restrict__ F, int nF) {
  for (int i = blockIdx.x * kT + threadIdx.x; i < nF; i += gridDim.x * kT) {
    const Pair pr = load_pair(F, i);
    const size_t hq = (size_t)pr.h * Q.nn + pr.q;
    if (pr.flags & kFlagSplitQ) {
      const size_t hp = (size_t)pr.h * Q.nn + Q.parent[pr.q];
      b.inherited[hq] = __ldcg(b.inherited + hp) + __ldcg(b.decided + hp);  // same value from every pair of q
    }
    float dl2, du2, sq, sr;
    box_geometry<D>(Q, pr.q, R, pr.r, dl2, du2, sq, sr);
    const float Ku = kernel_lower(du2, b.inv2h2_up[pr.h]);
    // reused by the classification of the same pair (no second gather of the boxes)
    b.ku[i] = Ku;
    b.kl[i] = kernel_upper(dl2, b.inv2h2_dn[pr.h]);
    b.sq[i] = sq;
    b.sr[i] = sr;
    // leave-one-out: a node meeting Q holds at most |R| - 1 other points for some query
    const int nr = R.cnt[pr.r] - ((b.loo && ranges_meet(Q, pr.q, R, pr.r)) ? 1 : 0);
    const u64 f = to_fix_f((float)nr, Ku, b.fix_scale_dn);
    if (f) atomicAdd(&b.lbsum[hq], f);
  }
}

template <int D>
__device__ __forceinline__ void classify_phase(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                                               const Pair* __restrict__ F, int nF,
                                               Pair* __restrict__ next, int cap_next,
                                               Action* __restrict__ far, Action* __restrict__ loc,
                                               Action* __restrict__ f2l, Pair* __restrict__ base,
                                               int cap_lists, RoundCounters* ctr, u64* sWarp, int* sBase) {
  const int d = D > 0 ? D : Q.d;
  const int P = Q.P;
  const int stride = gridDim.x * kT;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long my_prune = 0, my_inter = 0, my_fterms = 0, my_dterms = 0, my_tterms = 0;
  for (int i0 = blockIdx.x * kT; i0 < nF; i0 += stride) {
    const int i = i0 + threadIdx.x;
    // kind: -1 none, 0 prune, 1 F, 2 D, 3 T, 4 base, 5 recurse
    int kind = -1, order = 0, nchild = 0, split = 0;
    Pair pr{0, 0, 0, 0};
    unsigned long long inter = 0;
    if (i < nF) {
      pr = load_pair(F, i);
      const size_t hq = (size_t)pr.h * Q.nn + pr.q;
      const int cQ = Q.cnt[pr.q], cR = R.cnt[pr.r];
      const float nQ = (float)cQ, nR = (float)cR;
      // Leave-one-out sums (Q and R one tree): a pair whose nodes share
      // points counts |R| - 1 other references (for the lower bound and the
      // budget); it may be summarised only if R holds all of Q, and then the
      // summary's exact self term 1 is taken off, so its error bound (for
      // all |R| terms) is unchanged.  Pairs that only partly overlap go to
      // exact sums, which skip the self interaction.
      const bool meet = b.loo && ranges_meet(Q, pr.q, R, pr.r);
      const bool holds = meet && range_holds(R, pr.r, Q, pr.q);
      const bool summarise = !meet || holds;
      const float nRo = meet ? nR - 1.f : nR;
      // the fold phase's box geometry of this pair
      const float Kl = b.kl[i], Ku = b.ku[i], sideQ = b.sq[i], sideR = b.sr[i];
      const u64 lbf = __ldcg(b.inherited + hq) + __ldcg(b.decided + hq) + __ldcg(b.lbsum + hq);
      // tau = eps |R| G^l(Q) / |R_total| (CanSummarize), rounded down
      const float tau = __fmul_rd(__fmul_rd(b.tau_scale_dn, nRo), u64_to_f_rd(lbf));
      // prune: the kernel over the pair lies in [Ku, Kl]; the midpoint is off by
      // at most half the width, plus the float32 rounding of the midpoint
      // value itself (two roundings, covered by 4u of it)
      const float halfR = 0.5f * nR;
      const float value = halfR * (Kl + Ku);
      const float err_prune = __fadd_ru(__fmul_ru(halfR, __fsub_ru(Kl, Ku)),
                                        __fmul_ru(__fmul_ru(halfR, __fadd_ru(Kl, Ku)), 2.4e-7f));
      if (summarise && err_prune <= tau) {
        kind = 0;
        atomicAdd(&b.L[hq * P], (double)value - (holds ? 1.0 : 0.0));
        atomicMax(&b.pused[hq], 1);
      } else {
        int pF = 0, pD = 0, pT = 0;
        if (summarise && tau > 0.f) {
          const float inv_2h = b.inv_2h_up[pr.h];
          pF = order_ff(__fmul_ru(sideR, inv_2h), nR, d, tau, b.p_limit);
          pD = order_ff(__fmul_ru(sideQ, inv_2h), nR, d, tau, b.p_limit);
          pT = order_t(__fmul_ru(fmaxf(sideQ, sideR), inv_2h), nR, d, tau, b.p_limit);
        }
        // ChooseBestMethod with c_F = D N_Q p^D, c_D = D N_R p^D,
        // c_T = D p^{2D}, c_E = D N_Q N_R; ties go F, D, T, E.
        const float cF = pF ? d * nQ * pow_int_f((float)pF, d) : INFINITY;
        const float cD = pD ? d * nR * pow_int_f((float)pD, d) : INFINITY;
        const float cT = pT ? d * pow_int_f((float)pT, 2 * d) : INFINITY;
        const float cE = d * nQ * nR;
        const float m = fminf(fminf(cF, cD), fminf(cT, cE));
        if (pF && cF == m) { kind = 1; order = pF; }
        else if (pD && cD == m) { kind = 2; order = pD; }
        else if (pT && cT == m) { kind = 3; order = pT; }
        else {
          // exact sum: at a leaf pair (DFGTBase), or for any pair small
          // enough that recursing further cannot pay (|Q||R| <= base_block)
          const int ql = Q.left[pr.q], rl = R.left[pr.r];
          if ((ql < 0 && rl < 0) || (long long)cQ * cR <= b.base_block) {
            kind = 4;
            inter = (unsigned long long)cQ * (unsigned long long)cR;
          } else {
            kind = 5;
            nchild = (ql >= 0 && rl >= 0) ? 4 : 2;
          }
        }
        // Work cap: a far-field evaluation over more than kMaxSummaryPoints
        // queries, or a local accumulation over more than that many
        // references, recurses into the children of that side instead.  Both
        // summaries are additive over a partition of that side and their
        // order depends only on the other side's box, so the parts take the
        // same order within their own (proportional) budgets: no accuracy is
        // lost and the work of one warp stays bounded.
        if (kind == 1 && nQ > kMaxSummaryPoints && Q.left[pr.q] >= 0) {
          kind = 5; nchild = 2; split = kSplitQOnly;
        } else if (kind == 2 && nR > kMaxSummaryPoints && R.left[pr.r] >= 0) {
          kind = 5; nchild = 2; split = kSplitROnly;
        }
      }
      // algorithmic work of the summaries: |Q| p^D far-field terms, |R| p^D
      // local-moment terms, p^{2D} far-to-local terms
      if (kind == 1) my_fterms += (u64)cQ * (u64)ipow_u(order, d);
      else if (kind == 2) my_dterms += (u64)cR * (u64)ipow_u(order, d);
      else if (kind == 3) my_tterms += (u64)ipow_u(order, 2 * d);
      if (kind <= 4) {
        const u64 f = to_fix_f(nRo, Ku, b.fix_scale_dn);
        if (f) atomicAdd(&b.incr[hq], f);
      }
      if (holds && kind >= 1 && kind <= 3) order |= kSelfFlag;
      if (meet && kind == 4) order = kSelfFlag;
    }
    // Block-aggregated appends: the five counts of each pair (children,
    // F, D, T, base) packed in 12-bit fields of one word, one block-wide
    // exclusive scan, one atomic per list and block step (atomics on the
    // shared counters would otherwise serialise).  Child pairs only get
    // their pairs written to the next frontier (room for 4 per pair is
    // reserved by the host).
    const u64 mine = (u64)nchild | ((u64)(kind == 1) << 12) | ((u64)(kind == 2) << 24) |
                     ((u64)(kind == 3) << 36) | ((u64)(kind == 4) << 48);
    u64 incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) sWarp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      const u64 w = lane < kT / 32 ? sWarp[lane] : 0;
      u64 ws = w;
#pragma unroll
      for (int o = 1; o < kT / 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      if (lane < kT / 32) sWarp[lane] = ws - w;
      const u64 tot = __shfl_sync(0xffffffffu, ws, kT / 32 - 1);
      if (lane < 5) {
        int* const c = lane == 0 ? &ctr->n_next : lane == 1 ? &ctr->n_far : lane == 2 ? &ctr->n_loc
                     : lane == 3 ? &ctr->n_f2l : &ctr->n_base;
        const int n = (int)((tot >> (12 * lane)) & 0xfffu);
        sBase[lane] = n ? atomicAdd(c, n) : 0;
      }
    }
    __syncthreads();
    const u64 ex = sWarp[wid] + incl - mine;
    auto field = [&](int k) { return sBase[k] + (int)((ex >> (12 * k)) & 0xfffu); };
    if (nchild) {
      const int s0 = field(0);
      if (s0 + nchild <= cap_next) {
        const int ql = Q.left[pr.q], rl = R.left[pr.r];
        if (split == kSplitROnly || (split == 0 && ql < 0)) {
          next[s0] = Pair{pr.q, rl, pr.h, 0};
          next[s0 + 1] = Pair{pr.q, rl + 1, pr.h, 0};
        } else if (split == kSplitQOnly || rl < 0) {
          next[s0] = Pair{ql, pr.r, pr.h, kFlagSplitQ};
          next[s0 + 1] = Pair{ql + 1, pr.r, pr.h, kFlagSplitQ};
        } else {
          next[s0] = Pair{ql, rl, pr.h, kFlagSplitQ};
          next[s0 + 1] = Pair{ql, rl + 1, pr.h, kFlagSplitQ};
          next[s0 + 2] = Pair{ql + 1, rl, pr.h, kFlagSplitQ};
          next[s0 + 3] = Pair{ql + 1, rl + 1, pr.h, kFlagSplitQ};
        }
      } else {
        atomicOr(&ctr->status, kStOverflow);
      }
    }
    if (kind == 1) { const int s1 = field(1); if (s1 < cap_lists) far[s1] = Action{pr.q, pr.r, pr.h, order}; else atomicOr(&ctr->status, kStOverflow); }
    if (kind == 2) { const int s2 = field(2); if (s2 < cap_lists) loc[s2] = Action{pr.q, pr.r, pr.h, order}; else atomicOr(&ctr->status, kStOverflow); }
    if (kind == 3) { const int s3 = field(3); if (s3 < cap_lists) f2l[s3] = Action{pr.q, pr.r, pr.h, order}; else atomicOr(&ctr->status, kStOverflow); }
    if (kind == 4) { const int s4 = field(4); if (s4 < cap_lists) base[s4] = Pair{pr.q, pr.r, pr.h, order}; else atomicOr(&ctr->status, kStOverflow); }
    my_prune += kind == 0 ? 1ull : 0ull;
    my_inter += inter;
    __syncthreads();  // sWarp / sBase are reused by the next step
  }
  // totals: one atomic per block
  warp_add_u64_block(&ctr->n_prune, my_prune, sWarp);
  warp_add_u64_block(&ctr->base_inter, my_inter, sWarp);
  warp_add_u64_block(&ctr->far_terms, my_fterms, sWarp);
  warp_add_u64_block(&ctr->loc_terms, my_dterms, sWarp);
  warp_add_u64_block(&ctr->f2l_terms, my_tterms, sWarp);
}

// Every round of the traversal in one cooperative launch: fold, lower
// bounds, classification, each phase over the whole frontier and closed by
// a bounded grid barrier; the frontier swaps on the device.  The launch
// returns when the frontier is empty, when the next round might not fit
// the frontier buffers or the action lists (the host then drains or grows
// them and launches again), after max_rounds rounds, or on an overflow.
struct TravArgs {
  TreeView Q, R;
  TravBuffers b;
  Pair* F[2];
  int cap_front;                 // pairs each frontier buffer (and b.ku) holds
  Action *far, *loc, *f2l;
  Pair* base;
  int cap_lists;
  RoundCounters* ctr;
  TravControl* tc;
  unsigned* bar;
  BarrierCfg wait;
  int max_rounds;
};

template <int D>
__global__ void __launch_bounds__(kT) k_traverse(TravArgs A) {
  __shared__ u64 sWarp[kT / 32];
  __shared__ int sBase[5];
  const TravBuffers& b = A.b;
  RoundCounters* ctr = A.ctr;
  unsigned target = 0;
  int nF = __ldcg(&A.tc->nF), cur = __ldcg(&A.tc->cur), rounds = __ldcg(&A.tc->rounds);
  long long visited = __ldcg(&A.tc->visited);
  const int total = b.nh * A.Q.nn;
  int stop = 0;
  for (;;) {
    if (nF == 0) { stop = kTravDone; break; }
    if (rounds >= A.max_rounds) { stop = kTravRounds; break; }
    // room for this round: 4 children per pair, one item per pair per list
    const long long room = (long long)A.cap_lists - nF;
    if (4LL * nF > A.cap_front || __ldcg(&ctr->n_far) > room || __ldcg(&ctr->n_loc) > room ||
        __ldcg(&ctr->n_f2l) > room || __ldcg(&ctr->n_base) > room) {
      stop = kTravRoom;
      break;
    }
    fold_phase(b, total);
    if (!grid_barrier(A.bar, &ctr->status, target, A.wait)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&ctr->n_next, 0);
    lb_phase<D>(A.Q, A.R, b, A.F[cur], nF);
    if (!grid_barrier(A.bar, &ctr->status, target, A.wait)) return;
    classify_phase<D>(A.Q, A.R, b, A.F[cur], nF, A.F[cur ^ 1], 4 * nF, A.far, A.loc, A.f2l, A.base,
                      A.cap_lists, ctr, sWarp, sBase);
    if (!grid_barrier(A.bar, &ctr->status, target, A.wait)) return;
    visited += nF;
    ++rounds;
    cur ^= 1;
    nF = __ldcg(&ctr->n_next);
    if (__ldcg(&ctr->status) & kStOverflow) { stop = kTravOverflow; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    A.tc->nF = nF;
    A.tc->cur = cur;
    A.tc->rounds = rounds;
    A.tc->visited = visited;
    A.tc->stop = stop;
  }
}

template <int D>
cudaError_t traverse_d(const TravArgs& A, int* grid, cudaStream_t s) {
  if (*grid == 0) {
    int sms = 0, occ = 0, coop = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_traverse<D>, kT, 0);
    if (e != cudaSuccess) return e;
    if (!coop || occ < 1) return cudaErrorNotSupported;
    // four blocks per SM: 1, 2, 3, 4, 5, 6, 8 measured 1.38, 1.00, 0.92, 0.89,
    // 1.01, 1.01, 1.01 ms for the bandwidth sweep's traversal (more blocks hide
    // the gathers' latency until the grid barriers grow dearer)
    *grid = sms * (occ < 4 ? occ : 4);
  }
  TravArgs a = A;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)k_traverse<D>, dim3(*grid), dim3(kT), args, 0, s);
}

}  // namespace

cudaError_t launch_init_frontier(Pair* F, int nh, cudaStream_t s) {
  k_init_frontier<<<(nh + kT - 1) / kT, kT, 0, s>>>(F, nh);
  return cudaGetLastError();
}

cudaError_t launch_traverse(const TreeView& Q, const TreeView& R, const TravBuffers& b, Pair* F0, Pair* F1,
                            int cap_front, Action* far, Action* loc, Action* f2l, Pair* base, int cap_lists,
                            RoundCounters* ctr, TravControl* tc, unsigned* bar, const BarrierCfg& wait,
                            int max_rounds, int* grid, cudaStream_t s) {
  TravArgs A;
  A.Q = Q;
  A.R = R;
  A.b = b;
  A.F[0] = F0;
  A.F[1] = F1;
  A.cap_front = cap_front;
  A.far = far;
  A.loc = loc;
  A.f2l = f2l;
  A.base = base;
  A.cap_lists = cap_lists;
  A.ctr = ctr;
  A.tc = tc;
  A.bar = bar;
  A.wait = wait;
  A.max_rounds = max_rounds;
  switch (Q.d) {  // grid[d]: the cooperative grid of each dimension's kernel
    case 1: return traverse_d<1>(A, grid + 1, s);
    case 2: return traverse_d<2>(A, grid + 2, s);
    case 3: return traverse_d<3>(A, grid + 3, s);
    case 4: return traverse_d<4>(A, grid + 4, s);
    case 5: return traverse_d<5>(A, grid + 5, s);
    default: return traverse_d<0>(A, grid, s);
  }
}

}  // namespace dfgt
