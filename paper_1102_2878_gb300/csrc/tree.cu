// tree.cu -- device build of the mid-point kd-tree (Algorithm 2, BuildKdTree)
// and of the raw far-field moments of every node (Eq. far_field_moments at
// the leaves, the far-to-far translation of Lemma 3.5 upward).
//
// The build is level-synchronous, all levels in one persistent cooperative
// launch: every level has the tight bounding box of each of its nodes,
// splits the widest dimension at the box midpoint when the node holds more
// points than the leaf threshold, and stably partitions the points of
// every split node (x[sd] <= sc to the left) with one device-wide prefix
// sum.  Nodes are numbered level by level, so each level is a contiguous
// index range and the two children of a node are adjacent.  A split that
// would leave one side empty (all points equal along the widest side, or a
// midpoint that rounds onto the upper bound) turns the node into a leaf.
//
// Moments are kept unscaled, m_alpha = sum_r (r-c)^alpha / alpha!, in
// float64 about the box center c; the bandwidth scaling (2h^2)^(-|alpha|/2)
// of Eq. far_field_moments is applied where they are used, so one table
// serves every bandwidth.
#include <algorithm>
#include <cstring>

#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kT = 256;
constexpr int kMaxLevels = 128;
// Defaults measured on a GB300 (D = 3, 2e5 clustered points, 10 bandwidths
// in [1e-3, 1], eps = 1e-2): leaf sizes 16..256 and exact-sum thresholds
// 2048..65536 were timed; leaves of 128 points with pairs of up to 4096
// interactions summed exactly were fastest (17% faster than 32 / 4096).
// dfgt_autotune picks them per workload.
constexpr int kDefaultLeaf = 128;
constexpr long long kDefaultBaseBlock = 4096;

// The root: all points, no children; level 0 = [0, 1).  Its box is formed
// by the level build.
__global__ void k_init_root(int n, int* beg, int* cnt, int* left, int* parent, int* lv) {
  beg[0] = 0;
  cnt[0] = n;
  left[0] = -1;
  parent[0] = -1;
  lv[0] = 0;
  lv[1] = 1;
}

// ------------------------------------------------------------ level build
// All levels run in one cooperative launch: one block per SM, all
// co-resident, meeting at a grid barrier between the phases of a level.
// Block b owns a fixed slice of the point positions and, at every level, a
// slice of that level's nodes.  A level takes three phases:
//   1. each point of a node that splits is flagged when it goes left
//      (x[sd] <= sc); the flags are counted per block and per node;
//   2. the flags' device-wide exclusive prefix (the stable left rank of
//      every point) and each node's decision: it splits when the split rule
//      holds and both sides are non-empty, else it is a leaf;
//   3. children are numbered by the prefix of split decisions over the
//      level (so each level is a contiguous node range and siblings are
//      adjacent), the points are moved into their child's range in the
//      other point buffer, and the children's tight boxes are formed from
//      the moved points.
// The phases are latency-bound (a few dependent L2 round trips each), so a
// thread issues the loads of all its points before using any of them.  The
// launch ends when a level has no split, or when the next level would not
// fit the node arrays; then the host grows them and launches again at that
// level.
constexpr int kBT = 1024;       // threads per block of the level build
constexpr int kKB = 2;          // points per thread per pass
constexpr int kMaxGrid = 1024;  // blocks of the level build at most
constexpr long long kSpinLimit = 1LL << 25;  // barrier polls before giving up (~1 s)

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch on a monotone arrival counter:
// every block passes the same sequence of barriers, so the k-th barrier
// opens when the counter reaches k * gridDim.x (`target`, kept by each
// block).  The wait is bounded: a block that polls kSpinLimit times sets
// kStTimeout and leaves; every block returns false from then on, as it does
// once a non-finite coordinate has been seen.
__device__ bool grid_barrier(unsigned* bar, int* status, unsigned& target) {
  __shared__ int s_ok;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    long long it = 0;
    while ((int)(ld_acquire(bar) - target) < 0) {
      if (++it > kSpinLimit) {
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

// Exclusive prefix of v over the block's threads; `total` gets the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int& total, int* sw) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < kBT / 32 ? sw[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kBT / 32) sw[lane] = t;
  }
  __syncthreads();
  const int before = w > 0 ? sw[w - 1] : 0;
  total = sw[kBT / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// pre[0..G] = exclusive prefix of c[0..G) (and the total at pre[G]).
__device__ void grid_prefix(const int* c, int G, int* pre, int* sw) {
  int run = 0;
  for (int base = 0; base < G; base += kBT) {
    const int i = base + threadIdx.x;
    const int v = i < G ? __ldcg(c + i) : 0;
    int tot;
    const int ex = block_exclusive_scan(v, tot, sw);
    if (i < G) pre[i] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) pre[G] = run;
  __syncthreads();
}

// Split rule of node j: it splits only if it holds more than `leaf` points
// and its box has positive extent, along its widest side sd at the box
// midpoint sc (Algorithm 2).  Reads data other blocks wrote (L2 loads).
__device__ __forceinline__ bool split_rule(int j, int d, int leaf, const int* cnt, const float* lo,
                                           const float* hi, int& sd, float& sc) {
  sd = 0;
  float ext = __ldcg(hi + (size_t)j * d) - __ldcg(lo + (size_t)j * d);
  for (int k = 1; k < d; ++k) {
    const float x = __ldcg(hi + (size_t)j * d + k) - __ldcg(lo + (size_t)j * d + k);
    if (x > ext) { ext = x; sd = k; }
  }
  sc = 0.5f * (__ldcg(lo + (size_t)j * d + sd) + __ldcg(hi + (size_t)j * d + sd));
  return __ldcg(cnt + j) > leaf && ext > 0.f;
}

struct LevelArgs {
  const float* in;                  // caller's points [n][d]
  float *pbuf0, *pbuf1;             // padded points [n][dp], ping-pong
  int *perm0, *perm1;               // original index of each point
  int *pnode0, *pnode1;             // node of each point at the current level (-1: in a leaf)
  int* flag;                        // [n] goes left
  int* leftpos;                     // [n] exclusive prefix of flag
  int* bcnt;                        // [3 G] per block: flags, splits, leaves
  float *lo, *hi;                   // node boxes [cap][d]
  int *beg, *cnt, *left, *parent;   // node records [cap]
  int* nleft;                       // [cap] points going left
  int* lp0;                         // [cap] left prefix at the node's first point
  int* sloc;                        // [cap] split: rank among the block's splits; leaf: -1 - rank
  int* leaves;                      // [cap] leaf ids in node order
  int* lv;                          // level table: [3L] first node, [3L+1] end, [3L+2] splits
  int* ctl;                         // [0] status, [1] point buffer, [2] level, [3] leaves, [4] done, [5] nodes needed
  unsigned* bar;                    // grid barrier counter (zero at launch)
  int n, d, dp, leaf, cap, init_from, max_levels;
};

// Per-warp partial boxes of the children of one pass (phase 3).
struct WarpBox {
  int c0;         // left child of the warp's parent, or -1
  unsigned lr;    // bit 0: has left points, bit 1: has right points
};

__global__ void __launch_bounds__(kBT, 1) k_build_levels(LevelArgs A) {
  __shared__ int sw[kBT / 32];
  __shared__ int sPre[2][kMaxGrid + 1];
  __shared__ float sRed[2][kBT / 32];
  __shared__ WarpBox sWB[kBT / 32];
  __shared__ float sBox[kBT / 32][4][4];  // [warp][lmin, lmax, rmin, rmax][dimension, first 4]
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n = A.n, d = A.d, dp = A.dp;
  const int PC = (n + G - 1) / G;
  const int p0 = min(n, b * PC), p1 = min(n, p0 + PC);
  unsigned target = 0;
  int cur = __ldcg(A.ctl + 1), level = __ldcg(A.ctl + 2), nleaves = __ldcg(A.ctl + 3);

  // boxes and left counts of the nodes this launch may create
  for (size_t j = (size_t)A.init_from + (size_t)b * kBT + tid; j < (size_t)A.cap; j += (size_t)G * kBT) {
    A.nleft[j] = 0;
    for (int k = 0; k < d; ++k) {
      A.lo[j * d + k] = INFINITY;
      A.hi[j * d + k] = -INFINITY;
    }
  }
  if (!grid_barrier(A.bar, A.ctl, target)) return;

  if (A.init_from == 0) {
    // the root: padded copies of the points and its box
    bool bad = false;
    for (int i = p0 + tid; i < p1; i += kBT) {
      for (int k = 0; k < dp; ++k) {
        const float v = k < d ? A.in[(size_t)i * d + k] : 0.f;
        if (!isfinite(v)) bad = true;
        A.pbuf0[(size_t)i * dp + k] = v;
      }
      A.perm0[i] = i;
      A.pnode0[i] = 0;
    }
    if (bad) atomicOr(A.ctl, kStNonFinite);
    for (int k = 0; k < d; ++k) {
      float mn = INFINITY, mx = -INFINITY;
      for (int i = p0 + tid; i < p1; i += kBT) {
        const float v = A.in[(size_t)i * d + k];
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (lane == 0) { sRed[0][wid] = mn; sRed[1][wid] = mx; }
      __syncthreads();
      if (tid == 0 && p1 > p0) {
        for (int w = 1; w < kBT / 32; ++w) { mn = fminf(mn, sRed[0][w]); mx = fmaxf(mx, sRed[1][w]); }
        atomic_min_f(A.lo + k, mn);
        atomic_max_f(A.hi + k, mx);
      }
      __syncthreads();
    }
    if (!grid_barrier(A.bar, A.ctl, target)) return;
  }

  for (;;) {
    const int a = __ldcg(A.lv + 3 * level), e = __ldcg(A.lv + 3 * level + 1);
    const float* pin = cur ? A.pbuf1 : A.pbuf0;
    float* pout = cur ? A.pbuf0 : A.pbuf1;
    const int* permin = cur ? A.perm1 : A.perm0;
    int* permout = cur ? A.perm0 : A.perm1;
    const int* pnin = cur ? A.pnode1 : A.pnode0;
    int* pnout = cur ? A.pnode0 : A.pnode1;
    const int nn = e - a, NC = (nn + G - 1) / G;
    const int j0 = a + min(nn, b * NC), j1 = a + min(nn, b * NC + NC);

    // phase 1: left flags, counted per block and per node
    int nflag = 0;
    for (int c0 = p0; c0 < p1; c0 += kBT * kKB) {
      int nd[kKB], sd[kKB], f[kKB];
      float sc[kKB];
#pragma unroll
      for (int k = 0; k < kKB; ++k) {
        const int i = c0 + k * kBT + tid;
        nd[k] = i < p1 ? __ldcg(pnin + i) : -1;
      }
#pragma unroll
      for (int k = 0; k < kKB; ++k) f[k] = nd[k] >= 0 && split_rule(nd[k], d, A.leaf, A.cnt, A.lo, A.hi, sd[k], sc[k]);
#pragma unroll
      for (int k = 0; k < kKB; ++k) {
        const int i = c0 + k * kBT + tid;
        if (f[k]) f[k] = __ldcg(pin + (size_t)i * dp + sd[k]) <= sc[k] ? 1 : 0;
      }
#pragma unroll
      for (int k = 0; k < kKB; ++k) {
        const int i = c0 + k * kBT + tid;
        if (i < p1) A.flag[i] = f[k];
        nflag += f[k];
        const unsigned m = __ballot_sync(0xffffffffu, f[k]);
        if (f[k]) {
          const unsigned peers = __match_any_sync(m, nd[k]);
          if (lane == __ffs(peers) - 1) atomicAdd(A.nleft + nd[k], __popc(peers));
        }
      }
    }
    {
      int tot;
      block_exclusive_scan(nflag, tot, sw);
      if (tid == 0) A.bcnt[b] = tot;
    }
    if (!grid_barrier(A.bar, A.ctl, target)) return;

    // phase 2: left ranks of the points (and of each node's first point),
    // decisions of the nodes
    {
      int pre;
      block_exclusive_scan(tid < b ? __ldcg(A.bcnt + tid) : 0, pre, sw);  // G <= kBT
      int run = pre;
      for (int c0 = p0; c0 < p1; c0 += kBT * kKB) {
        int fk[kKB], nd[kKB], np[kKB];
#pragma unroll
        for (int k = 0; k < kKB; ++k) {
          const int i = c0 + k * kBT + tid;
          fk[k] = i < p1 ? A.flag[i] : 0;
          nd[k] = i < p1 ? __ldcg(pnin + i) : -1;
          np[k] = (i < p1 && i > 0) ? __ldcg(pnin + i - 1) : -2;
        }
#pragma unroll
        for (int k = 0; k < kKB; ++k) {
          const int i = c0 + k * kBT + tid;
          int tot;
          const int ex = block_exclusive_scan(fk[k], tot, sw);
          if (i < p1) {
            A.leftpos[i] = run + ex;
            if (nd[k] >= 0 && nd[k] != np[k]) A.lp0[nd[k]] = run + ex;
          }
          run += tot;
        }
      }
    }
    {
      int ns = 0, nl = 0;
      for (int base = j0; base < j1; base += kBT) {
        const int j = base + tid;
        int sp = 0, lf = 0;
        if (j < j1) {
          int sd;
          float sc;
          const bool want = split_rule(j, d, A.leaf, A.cnt, A.lo, A.hi, sd, sc);
          const int c = __ldcg(A.cnt + j), l = __ldcg(A.nleft + j);
          sp = (want && l > 0 && l < c) ? 1 : 0;
          lf = 1 - sp;
        }
        int ts, tl;
        const int es = block_exclusive_scan(sp, ts, sw);
        const int el = block_exclusive_scan(lf, tl, sw);
        if (j < j1) A.sloc[j] = sp ? ns + es : -1 - (nl + el);
        ns += ts;
        nl += tl;
      }
      if (tid == 0) {
        A.bcnt[G + b] = ns;
        A.bcnt[2 * G + b] = nl;
      }
    }
    if (!grid_barrier(A.bar, A.ctl, target)) return;

    // phase 3: children, leaves, scatter
    grid_prefix(A.bcnt + G, G, sPre[0], sw);
    grid_prefix(A.bcnt + 2 * G, G, sPre[1], sw);
    const int S = sPre[0][G], NL = sPre[1][G];
    if (S == 0) {
      // the last level: all of its nodes are leaves
      for (int j = j0 + tid; j < j1; j += kBT) A.leaves[nleaves + sPre[1][b] + (-1 - __ldcg(A.sloc + j))] = j;
      if (b == 0 && tid == 0) {
        A.lv[3 * level + 2] = 0;
        A.ctl[1] = cur;
        A.ctl[2] = level;
        A.ctl[3] = nleaves + NL;
        A.ctl[4] = 1;
        A.ctl[5] = e;
      }
      return;
    }
    const long long e2 = (long long)e + 2LL * S;
    if (e2 > A.cap || level + 1 >= A.max_levels) {
      // no room for the next level: undo this level's left counts and stop
      // here; the level is redone after the host has grown the node arrays
      for (int j = j0 + tid; j < j1; j += kBT) A.nleft[j] = 0;
      if (b == 0 && tid == 0) {
        A.ctl[1] = cur;
        A.ctl[2] = level;
        A.ctl[3] = nleaves;
        A.ctl[4] = 0;
        A.ctl[5] = (int)min(e2, (long long)INT32_MAX);
      }
      return;
    }
    for (int j = j0 + tid; j < j1; j += kBT) {
      const int s = __ldcg(A.sloc + j);
      if (s >= 0) {
        const int c0 = e + 2 * (sPre[0][b] + s);
        const int bg = __ldcg(A.beg + j), c = __ldcg(A.cnt + j), l = __ldcg(A.nleft + j);
        A.left[j] = c0;
        A.beg[c0] = bg;
        A.cnt[c0] = l;
        A.beg[c0 + 1] = bg + l;
        A.cnt[c0 + 1] = c - l;
        A.parent[c0] = A.parent[c0 + 1] = j;
        A.left[c0] = A.left[c0 + 1] = -1;
      } else {
        A.leaves[nleaves + sPre[1][b] + (-1 - s)] = j;
      }
    }
    if (b == 0 && tid == 0) {
      A.lv[3 * level + 2] = S;
      A.lv[3 * (level + 1)] = e;
      A.lv[3 * (level + 1) + 1] = (int)e2;
    }
    for (int c0 = p0; c0 < p1; c0 += kBT * kKB) {
      int nd[kKB], f[kKB], lpos[kKB], pm[kKB], s[kKB], b0[kKB], nl[kKB], l0[kKB];
#pragma unroll
      for (int k = 0; k < kKB; ++k) {
        const int i = c0 + k * kBT + tid;
        const bool in = i < p1;
        nd[k] = in ? __ldcg(pnin + i) : -1;
        f[k] = in ? A.flag[i] : 0;
        lpos[k] = in ? A.leftpos[i] : 0;
        pm[k] = in ? __ldcg(permin + i) : 0;
      }
#pragma unroll
      for (int k = 0; k < kKB; ++k) {
        s[k] = -1;
        b0[k] = nl[k] = l0[k] = 0;
        if (nd[k] >= 0) {
          s[k] = __ldcg(A.sloc + nd[k]);
          b0[k] = __ldcg(A.beg + nd[k]);
          nl[k] = __ldcg(A.nleft + nd[k]);
          l0[k] = __ldcg(A.lp0 + nd[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < kKB; ++k) {
        const int i = c0 + k * kBT + tid;
        const bool in = i < p1;
        int ch = -1, dst = i;
        if (s[k] >= 0) {
          const int cl = e + 2 * (sPre[0][(nd[k] - a) / NC] + s[k]);
          const int lrank = lpos[k] - l0[k];
          if (f[k]) {
            dst = b0[k] + lrank;
            ch = cl;
          } else {
            dst = b0[k] + nl[k] + (i - b0[k] - lrank);
            ch = cl + 1;
          }
        }
        if (in) {
          if ((unsigned)dst < (unsigned)n) {
            if (dp == 4) {
              const float4 v = __ldcg(reinterpret_cast<const float4*>(pin) + i);
              reinterpret_cast<float4*>(pout)[dst] = v;
            } else {
              for (int q = 0; q < dp; ++q) pout[(size_t)dst * dp + q] = __ldcg(pin + (size_t)i * dp + q);
            }
            permout[dst] = pm[k];
            pnout[dst] = ch;
          } else {
            atomicOr(A.ctl, kStOverflow);  // inconsistent ranks: never expected
            ch = -1;
          }
        }
        // children's boxes: a warp whose points share one parent (points are
        // contiguous per node) reduces with shuffles; the warps of the block
        // then merge runs of equal parents, so each child gets one atomic
        // per block and coordinate; other warps update per point
        const bool valid = in && ch >= 0;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        const int first = vm ? __ffs(vm) - 1 : 0;
        const int nd0 = __shfl_sync(0xffffffffu, nd[k], first);
        const int c00 = __shfl_sync(0xffffffffu, ch - (f[k] ? 0 : 1), first);
        const bool uni = vm != 0 && __all_sync(0xffffffffu, !valid || nd[k] == nd0);
        const unsigned lm = __ballot_sync(0xffffffffu, valid && f[k]), rm = vm & ~lm;
        if (lane == 0) {
          sWB[wid].c0 = uni ? c00 : -1;
          sWB[wid].lr = (lm ? 1u : 0u) | (rm ? 2u : 0u);
        }
        for (int q0 = 0; q0 < d; q0 += 4) {
          // up to four coordinates per round through shared memory
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const int q = q0 + qq;
            if (q >= d) break;
            const float v = valid ? __ldcg(pin + (size_t)i * dp + q) : 0.f;
            if (uni) {
              float lmn = (valid && f[k]) ? v : INFINITY, lmx = (valid && f[k]) ? v : -INFINITY;
              float rmn = (valid && !f[k]) ? v : INFINITY, rmx = (valid && !f[k]) ? v : -INFINITY;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                lmn = fminf(lmn, __shfl_xor_sync(0xffffffffu, lmn, o));
                lmx = fmaxf(lmx, __shfl_xor_sync(0xffffffffu, lmx, o));
                rmn = fminf(rmn, __shfl_xor_sync(0xffffffffu, rmn, o));
                rmx = fmaxf(rmx, __shfl_xor_sync(0xffffffffu, rmx, o));
              }
              if (lane == 0) {
                sBox[wid][0][qq] = lmn;
                sBox[wid][1][qq] = lmx;
                sBox[wid][2][qq] = rmn;
                sBox[wid][3][qq] = rmx;
              }
            } else if (valid) {
              atomic_min_f(A.lo + (size_t)ch * d + q, v);
              atomic_max_f(A.hi + (size_t)ch * d + q, v);
            }
          }
          __syncthreads();
          // thread (w, qq) of warp 0 .. : one thread per warp slot and
          // coordinate closes the run of equal parents that ends at its warp
          if (tid < (kBT / 32) * 4) {
            const int w = tid >> 2, qq = tid & 3, q = q0 + qq;
            const int cw = sWB[w].c0;
            const bool ends = cw >= 0 && q < d && (w == kBT / 32 - 1 || sWB[w + 1].c0 != cw);
            if (ends) {
              float lmn = INFINITY, lmx = -INFINITY, rmn = INFINITY, rmx = -INFINITY;
              unsigned lr = 0;
              for (int u = w; u >= 0 && sWB[u].c0 == cw; --u) {
                lmn = fminf(lmn, sBox[u][0][qq]);
                lmx = fmaxf(lmx, sBox[u][1][qq]);
                rmn = fminf(rmn, sBox[u][2][qq]);
                rmx = fmaxf(rmx, sBox[u][3][qq]);
                lr |= sWB[u].lr;
              }
              if (lr & 1u) {
                atomic_min_f(A.lo + (size_t)cw * d + q, lmn);
                atomic_max_f(A.hi + (size_t)cw * d + q, lmx);
              }
              if (lr & 2u) {
                atomic_min_f(A.lo + (size_t)(cw + 1) * d + q, rmn);
                atomic_max_f(A.hi + (size_t)(cw + 1) * d + q, rmx);
              }
            }
          }
          __syncthreads();
        }
      }
    }
    if (!grid_barrier(A.bar, A.ctl, target)) return;
    cur ^= 1;
    nleaves += NL;
    ++level;
  }
}

// ---------------------------------------------------------------- moments
// alpha digit of coefficient position idx (radix PM, last dimension least
// significant), matching the linear layout of the paper's appendix.
template <int D, int PM>
__device__ __forceinline__ int digit(int idx, int dd) {
  int v = idx;
  for (int k = D - 1; k > dd; --k) v /= PM;
  return v % PM;
}

// 1/n! for n < 16.
__constant__ double c_inv_fact[16] = {
    1.0, 1.0, 0.5, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720, 1.0 / 5040, 1.0 / 40320,
    1.0 / 362880, 1.0 / 3628800, 1.0 / 39916800, 1.0 / 479001600, 1.0 / 6227020800.0,
    1.0 / 87178291200.0, 1.0 / 1307674368000.0};

// Leaf moments (AccumulateFarFieldMoment): for each batch of 32 points the
// lanes tabulate the powers (r_k - c_k)^e, e < p_max, of one point each in
// shared memory; then each lane owns coefficient positions and accumulates
// prod_k table[j][k][alpha_k] over the batch.  Float64 throughout.
template <int D>
__global__ void __launch_bounds__(kT) k_leaf_moments(TreeView t, double* __restrict__ mom) {
  constexpr int PM = pmax_of(D);
  constexpr int P = ipow_c(PM, D);
  constexpr int S = (P + 31) / 32;
  constexpr int W = kT / 32;
  __shared__ double sPow[W][32][D][PM];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * W + wib;
  if (w >= t.nn || t.left[w] >= 0) return;
  double c[D];
#pragma unroll
  for (int k = 0; k < D; ++k) c[k] = 0.5 * ((double)t.lo[(size_t)w * D + k] + (double)t.hi[(size_t)w * D + k]);
  int al[S][D];
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    int v = lane + 32 * sl;
#pragma unroll
    for (int k = D - 1; k >= 0; --k) { al[sl][k] = v % PM; v /= PM; }
  }
  double acc[S];
#pragma unroll
  for (int sl = 0; sl < S; ++sl) acc[sl] = 0.0;
  const int b = t.beg[w], n = t.cnt[w];
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double x = j < n ? (double)t.pts[(size_t)(b + j) * t.dp + k] - c[k] : 0.0;
      double v = j < n ? 1.0 : 0.0;  // padding points contribute nothing
#pragma unroll
      for (int e = 0; e < PM; ++e) { sPow[wib][lane][k][e] = v; v *= x; }
    }
    __syncwarp();
    const int jn = min(32, n - j0);
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      if (lane + 32 * sl >= P) break;
      double a = 0.0;
      for (int jj = 0; jj < jn; ++jj) {
        double term = sPow[wib][jj][0][al[sl][0]];
#pragma unroll
        for (int k = 1; k < D; ++k) term *= sPow[wib][jj][k][al[sl][k]];
        a += term;
      }
      acc[sl] += a;
    }
    __syncwarp();
  }
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    const int idx = lane + 32 * sl;
    if (idx >= P) break;
    double f = 1.0;
#pragma unroll
    for (int k = 0; k < D; ++k) f *= c_inv_fact[al[sl][k]];
    mom[(size_t)w * P + idx] = acc[sl] * f;
  }
}

// Internal moments of one level by the far-to-far translation (Lemma 3.5,
// Eq. far_to_far_translation, exact for gamma < p) of both children:
// m_gamma(c') = sum_{alpha<=gamma} m_alpha(c_child) (c_child - c')^{gamma-alpha}/(gamma-alpha)!.
// The factor (x)^{gamma-alpha}/(gamma-alpha)! is a product over dimensions,
// so the shift is applied one dimension at a time (D p^D p operations per
// child instead of p^{2D}), in float64 shared memory, one warp per node.
template <int D>
__global__ void k_f2f_level(TreeView t, int a, int e, double* __restrict__ mom) {
  constexpr int PM = pmax_of(D);
  constexpr int P = ipow_c(PM, D);
  constexpr int W = kT / 32;
  __shared__ double sM[W][2][P];
  const int wib = threadIdx.x >> 5;
  const int w = a + blockIdx.x * W + wib;
  const int lane = threadIdx.x & 31;
  if (w >= e || t.left[w] < 0) return;
  double acc[(P + 31) / 32];
#pragma unroll
  for (int sl = 0; sl < (P + 31) / 32; ++sl) acc[sl] = 0.0;
  for (int ch = 0; ch < 2; ++ch) {
    const int cn = t.left[w] + ch;
    for (int idx = lane; idx < P; idx += 32) sM[wib][0][idx] = mom[(size_t)cn * P + idx];
    __syncwarp();
    int cur = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double x = 0.5 * ((double)t.lo[(size_t)cn * D + k] + (double)t.hi[(size_t)cn * D + k]) -
                       0.5 * ((double)t.lo[(size_t)w * D + k] + (double)t.hi[(size_t)w * D + k]);
      int stride = 1;
      for (int j = D - 1; j > k; --j) stride *= PM;
      double T[PM];  // x^e / e!
      T[0] = 1.0;
#pragma unroll
      for (int e2 = 1; e2 < PM; ++e2) T[e2] = T[e2 - 1] * x * (1.0 / (double)e2);
      for (int idx = lane; idx < P; idx += 32) {
        const int gk = (idx / stride) % PM;
        // sum over alpha_k <= gamma_k of m[.. alpha_k ..] x^{gamma_k - alpha_k} / (gamma_k - alpha_k)!
        double sum = 0.0;
#pragma unroll
        for (int dlt = 0; dlt < PM; ++dlt)
          if (dlt <= gk) sum += sM[wib][cur][idx - dlt * stride] * T[dlt];
        sM[wib][cur ^ 1][idx] = sum;
      }
      __syncwarp();
      cur ^= 1;
    }
#pragma unroll
    for (int sl = 0; sl < (P + 31) / 32; ++sl) {
      const int idx = lane + 32 * sl;
      if (idx < P) acc[sl] += sM[wib][cur][idx];
    }
    __syncwarp();
  }
#pragma unroll
  for (int sl = 0; sl < (P + 31) / 32; ++sl) {
    const int idx = lane + 32 * sl;
    if (idx < P) mom[(size_t)w * P + idx] = acc[sl];
  }
}

// Per-node float data for the float32 kernels: the box center as a float
// pair (hi + lo, so that differences with points stay accurate), the
// largest half side w and the moments normalised by w, m_alpha / w^|alpha|,
// which are bounded by |R| (each |r_k - c_k| <= w), so the scaled moments
// M_alpha = m~_alpha (w s)^|alpha| are formed in float32 without range
// problems.  Computed in float64 once per tree.
__global__ void k_node_float_data(TreeView t, int pm, float* __restrict__ chi, float* __restrict__ clo,
                                  float* __restrict__ whalf, float* __restrict__ mnorm) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= t.nn) return;
  const int d = t.d;
  double w = 0.0;
  for (int k = 0; k < d; ++k) {
    const double lo = t.lo[(size_t)j * d + k], hi = t.hi[(size_t)j * d + k];
    const double c = 0.5 * (lo + hi);
    const float h = (float)c;
    chi[(size_t)j * d + k] = h;
    clo[(size_t)j * d + k] = (float)(c - (double)h);
    w = fmax(w, 0.5 * (hi - lo));
  }
  float wf = (float)w;
  if (!(wf > 0.f)) wf = 1.f;
  whalf[j] = wf;
  const double iw = 1.0 / (double)wf;
  for (int idx = 0; idx < t.P; ++idx) {
    int v = idx, ab = 0;
    for (int k = 0; k < d; ++k) { ab += v % pm; v /= pm; }
    double sc = 1.0;
    for (int e = 0; e < ab; ++e) sc *= iw;
    mnorm[(size_t)j * t.P + idx] = (float)(t.mom[(size_t)j * t.P + idx] * sc);
  }
}

// D >= 6: p_max = 1, the only moment is m_0 = |R|.
__global__ void k_count_moments(TreeView t, double* __restrict__ mom) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < t.nn) mom[j] = (double)t.cnt[j];
}

template <int D>
cudaError_t moments_d(dfgt_tree* t, cudaStream_t s, long long* launches) {
  TreeView v = t->view();
  const int blocks = (int)(((size_t)t->nn * 32 + kT - 1) / kT);
  k_leaf_moments<D><<<blocks, kT, 0, s>>>(v, t->mom);
  ++*launches;
  for (int lev = t->depth - 2; lev >= 0; --lev) {
    const int a = t->lvl_off[lev], e = t->lvl_off[lev + 1];
    const int nb = (int)(((size_t)(e - a) * 32 + kT - 1) / kT);
    k_f2f_level<D><<<nb, kT, 0, s>>>(v, a, e, t->mom);
    ++*launches;
  }
  return cudaGetLastError();
}

// Node arrays of a build in progress, carved from one buffer with room
// for `cap` nodes.
struct NodeArrays {
  float *lo, *hi;
  int *beg, *cnt, *left, *parent, *nleft, *lp0, *sloc, *leaves;
  static size_t bytes(size_t cap, int d) {
    Carver c;
    NodeArrays a;
    a.carve(c, cap, d);
    return c.off;
  }
  void carve(Carver& c, size_t cap, int d) {
    lo = c.take<float>(cap * d);
    hi = c.take<float>(cap * d);
    beg = c.take<int>(cap);
    cnt = c.take<int>(cap);
    left = c.take<int>(cap);
    parent = c.take<int>(cap);
    nleft = c.take<int>(cap);
    lp0 = c.take<int>(cap);
    sloc = c.take<int>(cap);
    leaves = c.take<int>(cap);
  }
};

cudaError_t copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s, cudaError_t e) {
  if (e != cudaSuccess || bytes == 0) return e;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

// Grow the context's node buffer to `cap` nodes keeping the first `keep`
// nodes and the first `nleaves` leaf ids.
cudaError_t grow_nodes(DevBuf& buf, NodeArrays& na, size_t keep, size_t nleaves, size_t cap, int d,
                       cudaStream_t s) {
  DevBuf nb;
  cudaError_t e = nb.ensure(NodeArrays::bytes(cap, d));
  if (e != cudaSuccess) return e;
  Carver c{nb.as<char>()};
  NodeArrays nn;
  nn.carve(c, cap, d);
  e = copy_d2d(nn.lo, na.lo, keep * d * sizeof(float), s, e);
  e = copy_d2d(nn.hi, na.hi, keep * d * sizeof(float), s, e);
  e = copy_d2d(nn.beg, na.beg, keep * sizeof(int), s, e);
  e = copy_d2d(nn.cnt, na.cnt, keep * sizeof(int), s, e);
  e = copy_d2d(nn.left, na.left, keep * sizeof(int), s, e);
  e = copy_d2d(nn.parent, na.parent, keep * sizeof(int), s, e);
  e = copy_d2d(nn.nleft, na.nleft, keep * sizeof(int), s, e);
  e = copy_d2d(nn.leaves, na.leaves, nleaves * sizeof(int), s, e);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    nb.release();
    return e;
  }
  buf.release();
  buf = nb;
  na = nn;
  return cudaSuccess;
}

}  // namespace

void free_tree(dfgt_tree* t) {
  if (t->arena) {
    // every call on the tree has completed (calls return after their work),
    // so the arena can go back to the pool in any stream's order
    std::lock_guard<std::mutex> g(t->tpool->m);
    cudaFreeAsync(t->arena, t->tpool->stream);
  }
  t->arena = nullptr;
  t->tpool.reset();
  t->chi = t->clo = t->whalf = t->mnorm = nullptr;
  t->pts = nullptr; t->perm = nullptr; t->lo = t->hi = nullptr;
  t->beg = t->cnt = t->left = t->parent = t->leaves = nullptr; t->mom = nullptr;
}

#define TRY(x)                                                   \
  do {                                                           \
    cudaError_t _e = (x);                                        \
    if (_e != cudaSuccess) {                                     \
      ctx->err = std::string(#x) + ": " + cudaGetErrorString(_e); \
      goto fail;                                                 \
    }                                                            \
  } while (0)

dfgt_status build_tree(dfgt_ctx* ctx, const float* pts_dev, int64_t n64, int d,
                       const dfgt_opts* opts, dfgt_tree* t) {
  cudaStream_t s = ctx->stream;
  long long* L = &ctx->launches;
  const int n = (int)n64;
  t->n = n64;
  t->d = d;
  t->dp = padded_dim(d);
  t->leaf = (opts && opts->leaf_size > 0) ? opts->leaf_size : kDefaultLeaf;
  t->pm = pmax_of(d);
  t->P = ipow_c(t->pm, d);
  t->p_limit = (opts && opts->p_max > 0) ? std::min(opts->p_max, t->pm) : t->pm;
  t->eps_fp = (opts && opts->eps_fp > 0) ? opts->eps_fp : 2e-5;
  {
    const long long bb = opts ? opts->base_block : 0;
    t->base_block = bb > 0 ? bb : bb < 0 ? 0 : kDefaultBaseBlock;
  }
  t->lvl_off.assign(1, 0);

  // level-build scratch from the context: two point buffers, per-point node
  // ids, flags, left ranks, per-block counts, control words, the level table
  float* pbuf[2];
  int* perm2[2];
  int* pnode[2];
  int *flag, *leftpos, *bcnt, *ctl, *lv;
  unsigned* bar;
  NodeArrays na;
  size_t cap = 0;
  int cur = 0, last = -1;
  int h_ctl[8] = {};
  dfgt_status rc = DFGT_ECUDA;
  std::vector<int> lvh(3 * (kMaxLevels + 2));

  const size_t np = (size_t)n;
  Carver cv;
  for (int pass = 0; pass < 2; ++pass) {
    cv.off = 0;
    pbuf[0] = cv.take<float>(np * t->dp);
    pbuf[1] = cv.take<float>(np * t->dp);
    perm2[0] = cv.take<int>(np);
    perm2[1] = cv.take<int>(np);
    pnode[0] = cv.take<int>(np);
    pnode[1] = cv.take<int>(np);
    flag = cv.take<int>(np);
    leftpos = cv.take<int>(np);
    bcnt = cv.take<int>(3 * kMaxGrid);
    ctl = cv.take<int>(8);
    bar = cv.take<unsigned>(2);
    lv = cv.take<int>(3 * (kMaxLevels + 2));
    if (pass == 0) {
      TRY(ctx->bscratch.ensure(cv.off));
      cv.base = ctx->bscratch.as<char>();
    }
  }

  cap = std::max<size_t>(64, 4 * np / std::max(1, t->leaf) + 16);
  {
    TRY(ctx->bnodes.ensure(NodeArrays::bytes(cap, d)));
    // use all the room the buffer has
    const size_t fit = (ctx->bnodes.bytes - 10 * 256) / (8 * (size_t)d + 32);
    if (fit > cap && NodeArrays::bytes(fit, d) <= ctx->bnodes.bytes) cap = fit;
    Carver c{ctx->bnodes.as<char>()};
    na.carve(c, cap, d);
  }
  if (ctx->build_grid == 0) {
    // co-resident blocks of the level build: one per SM
    int coop = 0, sms = 0, occ = 0;
    TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
    TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_build_levels, kBT, 0));
    if (!coop || occ < 1) {
      ctx->err = "dfgt_build: the device does not support cooperative launches";
      goto fail;
    }
    ctx->build_grid = std::min(kMaxGrid, sms);
  }

  TRY(cudaMemsetAsync(ctl, 0, 8 * sizeof(int), s));
  k_init_root<<<1, 1, 0, s>>>(n, na.beg, na.cnt, na.left, na.parent, lv);
  ++*L;
  TRY(cudaGetLastError());
  {
    // One launch builds every level; it stops early only when the next
    // level would not fit the node arrays, which are then grown (each time
    // at least doubled) before the build goes on from that level.
    int init_from = 0;
    for (;;) {
      TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
      LevelArgs A;
      A.in = pts_dev;
      A.pbuf0 = pbuf[0]; A.pbuf1 = pbuf[1];
      A.perm0 = perm2[0]; A.perm1 = perm2[1];
      A.pnode0 = pnode[0]; A.pnode1 = pnode[1];
      A.flag = flag; A.leftpos = leftpos; A.bcnt = bcnt;
      A.lo = na.lo; A.hi = na.hi; A.beg = na.beg; A.cnt = na.cnt; A.left = na.left; A.parent = na.parent;
      A.nleft = na.nleft; A.lp0 = na.lp0; A.sloc = na.sloc; A.leaves = na.leaves;
      A.lv = lv; A.ctl = ctl; A.bar = bar;
      A.n = n; A.d = d; A.dp = t->dp; A.leaf = t->leaf;
      A.cap = (int)std::min<size_t>(cap, INT32_MAX);
      A.init_from = init_from;
      A.max_levels = kMaxLevels;
      void* args[] = {&A};
      TRY(cudaLaunchCooperativeKernel((const void*)k_build_levels, dim3(ctx->build_grid), dim3(kBT), args, 0, s));
      ++*L;
      TRY(cudaMemcpyAsync(h_ctl, ctl, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(cudaMemcpyAsync(lvh.data(), lv, lvh.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(cudaStreamSynchronize(s));
      if (h_ctl[0] & kStNonFinite) {
        ctx->err = "dfgt_build: non-finite coordinate";
        rc = DFGT_EINVAL;
        goto fail;
      }
      if (h_ctl[0] & kStOverflow) {
        ctx->err = "dfgt_build: point rank out of range (internal error)";
        rc = DFGT_ECAPACITY;
        goto fail;
      }
      if (h_ctl[0] & kStTimeout) {
        ctx->err = "dfgt_build: a grid barrier wait timed out";
        rc = DFGT_ETIMEOUT;
        goto fail;
      }
      if (h_ctl[4]) break;
      const int level = h_ctl[2];
      if (level + 1 >= kMaxLevels) {
        ctx->err = "dfgt_build: more than 128 tree levels";
        rc = DFGT_ETIMEOUT;
        goto fail;
      }
      const size_t keep = (size_t)lvh[3 * level + 1];
      const size_t need = (size_t)h_ctl[5];
      if (need <= cap) {
        ctx->err = "dfgt_build: level build stopped without cause (internal error)";
        rc = DFGT_ECAPACITY;
        goto fail;
      }
      const size_t nc = std::max(need + need / 2, cap * 2);
      TRY(grow_nodes(ctx->bnodes, na, keep, (size_t)h_ctl[3], nc, d, s));
      cap = nc;
      init_from = (int)keep;
    }
    cur = h_ctl[1];
    last = h_ctl[2];
    t->nleaves = h_ctl[3];
    t->lvl_off.assign(1, 0);
    for (int Lk = 0; Lk <= last; ++Lk) t->lvl_off.push_back(lvh[3 * Lk + 1]);
  }
  t->nn = t->lvl_off.back();
  t->depth = (int)t->lvl_off.size() - 1;
  if (t->nn >= (1 << 27)) {  // node indices share a word with a 4-bit order in the sorted lists
    ctx->err = "dfgt_build: more than 2^27 tree nodes (raise leaf_size)";
    rc = DFGT_ECAPACITY;
    goto fail;
  }
  {
    // the tree's arena: one allocation from the context's pool
    const size_t nn = (size_t)t->nn, P = (size_t)t->P;
    Carver ca;
    for (int pass = 0; pass < 2; ++pass) {
      ca.off = 0;
      t->pts = ca.take<float>(np * t->dp);
      t->perm = ca.take<int>(np);
      t->leaves = ca.take<int>(nn);
      t->lo = ca.take<float>(nn * d);
      t->hi = ca.take<float>(nn * d);
      t->beg = ca.take<int>(nn);
      t->cnt = ca.take<int>(nn);
      t->left = ca.take<int>(nn);
      t->parent = ca.take<int>(nn);
      t->mom = ca.take<double>(nn * P);
      t->chi = ca.take<float>(nn * d);
      t->clo = ca.take<float>(nn * d);
      t->whalf = ca.take<float>(nn);
      t->mnorm = ca.take<float>(nn * P);
      if (pass == 0) {
        t->tpool = ctx->tpool;
        TRY(cudaMallocFromPoolAsync(&t->arena, ca.off, ctx->tpool->pool, s));
        ca.base = static_cast<char*>(t->arena);
      }
    }
    cudaError_t ce = cudaSuccess;
    ce = copy_d2d(t->pts, pbuf[cur], np * t->dp * sizeof(float), s, ce);
    ce = copy_d2d(t->perm, perm2[cur], np * sizeof(int), s, ce);
    ce = copy_d2d(t->lo, na.lo, nn * d * sizeof(float), s, ce);
    ce = copy_d2d(t->hi, na.hi, nn * d * sizeof(float), s, ce);
    ce = copy_d2d(t->beg, na.beg, nn * sizeof(int), s, ce);
    ce = copy_d2d(t->cnt, na.cnt, nn * sizeof(int), s, ce);
    ce = copy_d2d(t->left, na.left, nn * sizeof(int), s, ce);
    ce = copy_d2d(t->parent, na.parent, nn * sizeof(int), s, ce);
    ce = copy_d2d(t->leaves, na.leaves, (size_t)t->nleaves * sizeof(int), s, ce);
    TRY(ce);
  }
  switch (d) {
    case 1: TRY(moments_d<1>(t, s, L)); break;
    case 2: TRY(moments_d<2>(t, s, L)); break;
    case 3: TRY(moments_d<3>(t, s, L)); break;
    case 4: TRY(moments_d<4>(t, s, L)); break;
    case 5: TRY(moments_d<5>(t, s, L)); break;
    default:
      k_count_moments<<<(t->nn + kT - 1) / kT, kT, 0, s>>>(t->view(), t->mom);
      ++*L;
      TRY(cudaGetLastError());
  }
  k_node_float_data<<<(t->nn + kT - 1) / kT, kT, 0, s>>>(t->view(), t->pm, t->chi, t->clo, t->whalf, t->mnorm);
  ++*L;
  TRY(cudaGetLastError());
  TRY(cudaStreamSynchronize(s));  // calls return after their work
  rc = DFGT_OK;
fail:
  if (rc != DFGT_OK) {
    cudaStreamSynchronize(s);
    free_tree(t);
  }
  return rc;
}

}  // namespace dfgt
