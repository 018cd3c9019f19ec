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
  int* arrive;                      // [cap] moment-pass child counters (zeroed here)
  int* lp0;                         // [cap] left prefix at the node's first point
  int* sloc;                        // [cap] split: rank among the block's splits; leaf: -1 - rank
  int* leaves;                      // [cap] leaf ids in node order
  int* lv;                          // level table: [3L] first node, [3L+1] end, [3L+2] splits
  int* ctl;                         // [0] status, [1] point buffer, [2] level, [3] leaves, [4] done, [5] nodes needed
  unsigned* bar;                    // grid barrier counter (zero at launch)
  BarrierCfg wait;                  // how its waits are bounded
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
    A.arrive[j] = 0;
    for (int k = 0; k < d; ++k) {
      A.lo[j * d + k] = INFINITY;
      A.hi[j * d + k] = -INFINITY;
    }
  }
  if (!grid_barrier(A.bar, A.ctl, target, A.wait)) return;

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
    if (!grid_barrier(A.bar, A.ctl, target, A.wait)) return;
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
    if (!grid_barrier(A.bar, A.ctl, target, A.wait)) return;

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
    if (!grid_barrier(A.bar, A.ctl, target, A.wait)) return;

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
          float vq[4];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) vq[qq] = (valid && q0 + qq < d) ? __ldcg(pin + (size_t)i * dp + q0 + qq) : 0.f;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const int q = q0 + qq;
            if (q >= d) break;
            const float v = vq[qq];
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
    if (!grid_barrier(A.bar, A.ctl, target, A.wait)) return;
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

constexpr int kMT = 256;  // threads per block of the moment pass
constexpr int kMW = kMT / 32;

struct MomArgs {
  const float *pbuf0, *pbuf1;  // the level build's point buffers (ctl[1] holds the final one)
  const float *lo, *hi;
  const int *beg, *cnt, *left, *parent, *leaves;
  double* mom;                 // [nodes][P] raw moments
  float *chi, *clo, *whalf, *mnorm, *rad;
  int* arrive;                 // [nodes] children finished (zero at launch)
  const int* ctl;
  int n, d, dp, pm, P;
};

// Shared memory of one warp: a batch of 32 points' coordinate powers
// (leaf moments) or the moment buffers of a dimension-wise shift (F2F).
template <int D, int PM, int P>
union MomSmem {
  double pw[32][D][PM];
  double m[3][P];
};

// Leaf moments (AccumulateFarFieldMoment) of leaf w, one warp, float64:
// the points' powers (r_k - c_k)^e, e < p_max, are tabulated 32 points at
// a time; lane (g, pre) owns the digits alpha_0..alpha_{D-2} = pre and all
// p_max values of the last digit, and sums over every R-th point of the
// batch (R = 32 / p_max^{D-1} lane groups), so a term costs one multiply
// per leading digit and one FMA per last digit.
template <int D, int PM, int P>
__device__ void leaf_moments(const MomArgs& M, const float* pin, int w, MomSmem<D, PM, P>& sm) {
  constexpr int NPRE = P / PM;
  constexpr int R = 32 / NPRE;
  const int lane = threadIdx.x & 31, g = lane / NPRE, pre = lane % NPRE;
  double c[D];
#pragma unroll
  for (int k = 0; k < D; ++k) c[k] = 0.5 * ((double)M.lo[(size_t)w * D + k] + (double)M.hi[(size_t)w * D + k]);
  int al[D > 1 ? D - 1 : 1];
#pragma unroll
  for (int k = D - 2, v = pre; k >= 0; --k) { al[k] = v % PM; v /= PM; }
  double acc[PM];
#pragma unroll
  for (int e = 0; e < PM; ++e) acc[e] = 0.0;
  const int b = M.beg[w], n = M.cnt[w];
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int j = j0 + lane;
    float xr[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xr[k] = j < n ? pin[(size_t)(b + j) * M.dp + k] : 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double x = j < n ? (double)xr[k] - c[k] : 0.0;
      double v = 1.0;
#pragma unroll
      for (int e = 0; e < PM; ++e) { sm.pw[lane][k][e] = v; v *= x; }
    }
    __syncwarp();
    const int jn = min(32, n - j0);
    if (g < R) {
      for (int jj = g; jj < jn; jj += R) {
        double t = 1.0;
#pragma unroll
        for (int k = 0; k < D - 1; ++k) t *= sm.pw[jj][k][al[k]];
#pragma unroll
        for (int e = 0; e < PM; ++e) acc[e] = fma(t, sm.pw[jj][D - 1][e], acc[e]);
      }
    }
    __syncwarp();
  }
  // lanes of group 0 collect the other groups' sums (fixed order)
#pragma unroll
  for (int e = 0; e < PM; ++e) {
    double s = acc[e];
    for (int g2 = 1; g2 < R; ++g2) s += __shfl_sync(0xffffffffu, acc[e], (lane + g2 * NPRE) & 31);
    acc[e] = s;
  }
  if (g == 0) {
    double f = 1.0;
#pragma unroll
    for (int k = 0; k < D - 1; ++k) f *= c_inv_fact[al[k]];
#pragma unroll
    for (int e = 0; e < PM; ++e) M.mom[(size_t)w * P + pre * PM + e] = acc[e] * f * c_inv_fact[e];
  }
}

// Moments of internal node w by the far-to-far translation (Lemma 3.5,
// Eq. far_to_far_translation, exact for gamma < p) of both children:
// m_gamma(c') = sum_{alpha<=gamma} m_alpha(c_child) (c_child - c')^{gamma-alpha}/(gamma-alpha)!.
// The factor (x)^{gamma-alpha}/(gamma-alpha)! is a product over dimensions,
// so the shift is applied one dimension at a time (D p^D p operations per
// child instead of p^{2D}), in float64 shared memory, one warp per node.
// Every global load is issued before the arithmetic.
template <int D, int PM, int P>
__device__ void f2f_node(const MomArgs& M, int w, MomSmem<D, PM, P>& sm) {
  constexpr int S = (P + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int c0 = M.left[w];
  float lo3[3][D], hi3[3][D];
  double mv[2][S];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    lo3[0][k] = M.lo[(size_t)w * D + k];
    hi3[0][k] = M.hi[(size_t)w * D + k];
    lo3[1][k] = M.lo[(size_t)c0 * D + k];
    hi3[1][k] = M.hi[(size_t)c0 * D + k];
    lo3[2][k] = M.lo[(size_t)(c0 + 1) * D + k];
    hi3[2][k] = M.hi[(size_t)(c0 + 1) * D + k];
  }
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      const int idx = lane + 32 * sl;
      mv[ch][sl] = idx < P ? __ldcg(M.mom + (size_t)(c0 + ch) * P + idx) : 0.0;
    }
  double acc[S];
#pragma unroll
  for (int sl = 0; sl < S; ++sl) acc[sl] = 0.0;
#pragma unroll
  for (int ch = 0; ch < 2; ++ch) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      const int idx = lane + 32 * sl;
      if (idx < P) sm.m[0][idx] = mv[ch][sl];
    }
    __syncwarp();
    int cur = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double x = 0.5 * ((double)lo3[1 + ch][k] + (double)hi3[1 + ch][k]) -
                       0.5 * ((double)lo3[0][k] + (double)hi3[0][k]);
      int stride = 1;
#pragma unroll
      for (int j = D - 1; j > k; --j) stride *= PM;
      double T[PM];  // x^e / e!
      T[0] = 1.0;
#pragma unroll
      for (int e2 = 1; e2 < PM; ++e2) T[e2] = T[e2 - 1] * x * (1.0 / (double)e2);
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        const int idx = lane + 32 * sl;
        if (idx < P) {
          const int gk = (idx / stride) % PM;
          double sum = 0.0;
#pragma unroll
          for (int dlt = 0; dlt < PM; ++dlt)
            if (dlt <= gk) sum += sm.m[cur][idx - dlt * stride] * T[dlt];
          sm.m[cur ^ 1][idx] = sum;
        }
      }
      __syncwarp();
      cur ^= 1;
    }
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      const int idx = lane + 32 * sl;
      if (idx < P) acc[sl] += sm.m[cur][idx];
    }
    __syncwarp();
  }
#pragma unroll
  for (int sl = 0; sl < S; ++sl) {
    const int idx = lane + 32 * sl;
    if (idx < P) M.mom[(size_t)w * P + idx] = acc[sl];
  }
}

// Per-node float data for the float32 kernels, one warp: the box center as
// a float pair (hi + lo, so that differences with points stay accurate),
// the largest half side w and the moments normalised by w,
// m_alpha / w^|alpha|, which are bounded by |R| (each |r_k - c_k| <= w), so
// the scaled moments M_alpha = m~_alpha (w s)^|alpha| are formed in float32
// without range problems.  Computed in float64 once per tree; the node's
// moments were written by this warp or are visible to it.
__device__ void node_float_data(const MomArgs& M, const float* pin, int j) {
  const int d = M.d, lane = threadIdx.x & 31;
  double hw = 0.0;
  for (int k = lane; k < d; k += 32) {
    const double lo = M.lo[(size_t)j * d + k], hi = M.hi[(size_t)j * d + k];
    const double c = 0.5 * (lo + hi);
    const float h = (float)c;
    M.chi[(size_t)j * d + k] = h;
    M.clo[(size_t)j * d + k] = (float)(c - (double)h);
    hw = fmax(hw, 0.5 * (hi - lo));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hw = fmax(hw, __shfl_xor_sync(0xffffffffu, hw, o));
  // radius of the node's points about the float box centre 0.5f (lo + hi)
  // (the centre the distance bounds take), rounded up: a leaf from its
  // points, a parent from its children (|c - c_child| + r_child) or the box's
  // half diagonal, whichever is smaller
  float r2 = 0.f;
  const int left = M.left[j];
  if (left < 0) {
    const int b = M.beg[j], c = M.cnt[j];
    for (int i = lane; i < c; i += 32) {
      const float* p = pin + (size_t)(b + i) * M.dp;
      float s = 0.f;
      for (int k = 0; k < d; ++k) {
        const float ck = 0.5f * (M.lo[(size_t)j * d + k] + M.hi[(size_t)j * d + k]);
        const float v = p[k];
        const float df = v >= ck ? __fsub_ru(v, ck) : __fsub_ru(ck, v);
        s = __fmaf_ru(df, df, s);
      }
      r2 = fmaxf(r2, s);
    }
  } else {
    if (lane < 2) {
      const int ch = left + lane;
      float s = 0.f;
      for (int k = 0; k < d; ++k) {
        const float ck = 0.5f * (M.lo[(size_t)j * d + k] + M.hi[(size_t)j * d + k]);
        const float cc = 0.5f * (M.lo[(size_t)ch * d + k] + M.hi[(size_t)ch * d + k]);
        const float df = cc >= ck ? __fsub_ru(cc, ck) : __fsub_ru(ck, cc);
        s = __fmaf_ru(df, df, s);
      }
      const float r = __fadd_ru(__fsqrt_ru(s), __ldcg(M.rad + ch));
      r2 = __fmul_ru(r, r);
    }
  }
  // the box's half diagonal bounds it too
  float hd2 = 0.f;
  for (int k = lane; k < d; k += 32) {
    const float ck = 0.5f * (M.lo[(size_t)j * d + k] + M.hi[(size_t)j * d + k]);
    const float w = fmaxf(__fsub_ru(M.hi[(size_t)j * d + k], ck), __fsub_ru(ck, M.lo[(size_t)j * d + k]));
    hd2 = __fmaf_ru(w, w, hd2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, o));
    hd2 = __fadd_ru(hd2, __shfl_xor_sync(0xffffffffu, hd2, o));
  }
  if (lane == 0) M.rad[j] = fminf(__fsqrt_ru(r2), __fsqrt_ru(hd2));
  float wf = (float)hw;
  if (!(wf > 0.f)) wf = 1.f;
  if (lane == 0) M.whalf[j] = wf;
  const double iw = 1.0 / (double)wf;
  for (int idx = lane; idx < M.P; idx += 32) {
    const double m = __ldcg(M.mom + (size_t)j * M.P + idx);
    int v = idx, ab = 0;
    for (int k = 0; k < d; ++k) { ab += v % M.pm; v /= M.pm; }
    double sc = 1.0;
    for (int e = 0; e < ab; ++e) sc *= iw;
    M.mnorm[(size_t)j * M.P + idx] = (float)(m * sc);
  }
}

// Every moment of the tree, after the level build has finished (it returns
// at once otherwise): each warp sums the moments of its leaves, and the
// warp that finishes the second
// child of a node translates both children's moments to it (Lemma 3.5) and
// goes on up, so no warp waits for another.  Each node's float data follows
// its moments.  D = 0 stands for D >= 6, where p_max = 1 and the only
// moment is m_0 = |R|.
template <int D>
__global__ void __launch_bounds__(kMT) k_moments(MomArgs M) {
  constexpr int PM = D > 0 ? pmax_of(D) : 1;
  constexpr int P = D > 0 ? ipow_c(PM, D) : 1;
  constexpr int DD = D > 0 ? D : 1;
  __shared__ MomSmem<DD, PM, P> sm[kMW];
  if (__ldcg(M.ctl + 4) == 0) return;
  const int G = gridDim.x, wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kMW + wib, nw = G * kMW;
  const int cur = __ldcg(M.ctl + 1), nleaves = __ldcg(M.ctl + 3);
  const float* pin = cur ? M.pbuf1 : M.pbuf0;
  for (int li = gw; li < nleaves; li += nw) {
    int w = M.leaves[li];
    if constexpr (D > 0) {
      leaf_moments<D, PM, P>(M, pin, w, sm[wib]);
    } else {
      if (lane == 0) M.mom[w] = (double)M.cnt[w];
    }
    __syncwarp();
    node_float_data(M, pin, w);
    for (;;) {
      const int par = M.parent[w];
      if (par < 0) break;
      // publish this node's moments, then count it as a finished child
      __threadfence();
      int prev = 0;
      if (lane == 0) prev = atomicAdd(M.arrive + par, 1);
      prev = __shfl_sync(0xffffffffu, prev, 0);
      if (prev == 0) break;  // the sibling's warp will do the parent
      __threadfence();
      if constexpr (D > 0) {
        f2f_node<D, PM, P>(M, par, sm[wib]);
      } else {
        if (lane == 0) M.mom[par] = (double)M.cnt[par];
      }
      __syncwarp();
      node_float_data(M, pin, par);
      w = par;
    }
  }
}

cudaError_t copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s, cudaError_t e) {
  if (e != cudaSuccess || bytes == 0) return e;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

// The tree's arena: one pool allocation holding every array of the tree,
// with room for `cap` nodes.  The level build writes the node records into
// it directly.
void carve_tree(Carver& ca, dfgt_tree* t, size_t np, size_t cap) {
  const int d = t->d;
  const size_t P = (size_t)t->P;
  t->pts = ca.take<float>(np * t->dp);
  t->perm = ca.take<int>(np);
  t->leaves = ca.take<int>(cap);
  t->lo = ca.take<float>(cap * d);
  t->hi = ca.take<float>(cap * d);
  t->beg = ca.take<int>(cap);
  t->cnt = ca.take<int>(cap);
  t->left = ca.take<int>(cap);
  t->parent = ca.take<int>(cap);
  t->mom = ca.take<double>(cap * P);
  t->chi = ca.take<float>(cap * d);
  t->clo = ca.take<float>(cap * d);
  t->whalf = ca.take<float>(cap);
  t->mnorm = ca.take<float>(cap * P);
  t->rad = ca.take<float>(cap);
}

cudaError_t alloc_tree(dfgt_ctx* ctx, dfgt_tree* t, size_t np, size_t cap) {
  Carver ca;
  dfgt_tree shape;  // sizes only; t keeps its arrays if the allocation fails
  shape.d = t->d;
  shape.dp = t->dp;
  shape.P = t->P;
  carve_tree(ca, &shape, np, cap);
  void* arena = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&arena, ca.off, ctx->tpool->pool, ctx->stream);
  if (e != cudaSuccess) return e;
  t->tpool = ctx->tpool;
  t->arena = arena;
  Carver cb{static_cast<char*>(arena)};
  carve_tree(cb, t, np, cap);
  return cudaSuccess;
}

// Per-node scratch of the level build in the context (left counts, moment
// pass counters, left prefixes, split ranks), `cap` nodes each.
struct NodeScratch {
  int *nleft, *arrive, *lp0, *sloc;
  static size_t bytes(size_t cap) { return 4 * ((cap * sizeof(int) + 255) & ~(size_t)255) + 256; }
  void carve(char* base, size_t cap) {
    Carver c{base};
    nleft = c.take<int>(cap);
    arrive = c.take<int>(cap);
    lp0 = c.take<int>(cap);
    sloc = c.take<int>(cap);
  }
};

// Blocks of a cooperative launch of `fn`: `per_sm` per SM at most.
template <class F>
cudaError_t coop_grid(F fn, int threads, int per_sm, int device, int* grid) {
  int coop = 0, sms = 0, occ = 0;
  cudaError_t e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0);
  if (e != cudaSuccess) return e;
  if (!coop || occ < 1) return cudaErrorNotSupported;
  *grid = std::min(kMaxGrid, sms * std::min(occ, per_sm));
  return cudaSuccess;
}

template <int D>
cudaError_t launch_moments(dfgt_ctx* ctx, const MomArgs& M, cudaStream_t s) {
  int& g = ctx->mom_grid[D];
  if (g == 0) {
    int sms = 0;
    const cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return e;
    g = 4 * sms;
  }
  k_moments<D><<<g, kMT, 0, s>>>(M);
  return cudaGetLastError();
}

}  // namespace

void free_tree(dfgt_tree* t) {
  if (t->arena) {
    // every call on the tree has completed (calls return after their work)
    // but the build's moment pass may still run: the arena goes back to the
    // pool after it, in the pool stream's order
    std::lock_guard<std::mutex> g(t->tpool->m);
    if (t->ready) {
      if (t->tpool->stream)
        cudaStreamWaitEvent(t->tpool->stream, t->ready, 0);
      else
        cudaEventSynchronize(t->ready);
    }
    cudaFreeAsync(t->arena, t->tpool->stream);
  }
  if (t->ready) cudaEventDestroy(t->ready);
  t->ready = nullptr;
  for (cudaEvent_t& e : t->tev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  t->arena = nullptr;
  t->tpool.reset();
  t->chi = t->clo = t->whalf = t->mnorm = t->rad = nullptr;
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
  t->eps_fp = (opts && opts->eps_fp > 0) ? opts->eps_fp : 0.0;  // 0: chosen per sum from eps
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
  NodeScratch ns;
  size_t cap = 0;
  int h_ctl[8] = {};
  dfgt_status rc = DFGT_ECUDA;
  std::vector<int> lvh(3 * (kMaxLevels + 2));

  const size_t np = (size_t)n;
  Carver cv;
  // the previous build's moment pass may still read the build scratch
  TRY(cudaStreamWaitEvent(s, ctx->moments_done, 0));
  TRY(cudaEventCreateWithFlags(&t->ready, cudaEventDisableTiming));
  for (cudaEvent_t& e : t->tev) TRY(cudaEventCreate(&e));
  TRY(cudaEventRecord(t->tev[0], s));
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
  if (ctx->build_grid == 0) {
    const cudaError_t e = coop_grid(k_build_levels, kBT, 1, ctx->device, &ctx->build_grid);
    if (e == cudaErrorNotSupported) {
      ctx->err = "dfgt_build: the device does not support cooperative launches";
      goto fail;
    }
    TRY(e);
  }

  // node capacity: a level has at most 2 floor(n / (leaf + 1)) nodes below
  // the root; twice that covers typical trees, and the build grows it
  cap = std::max<size_t>(64, 4 * np / std::max(1, t->leaf) + 16);
  TRY(alloc_tree(ctx, t, np, cap));
  TRY(ctx->bnodes.ensure(NodeScratch::bytes(cap)));
  ns.carve(ctx->bnodes.as<char>(), cap);

  TRY(cudaMemsetAsync(ctl, 0, 8 * sizeof(int), s));
  k_init_root<<<1, 1, 0, s>>>(n, t->beg, t->cnt, t->left, t->parent, lv);
  ++*L;
  TRY(cudaGetLastError());
  {
    // One launch builds every level and one more forms every moment; the
    // level build stops early only when the next level would not fit the
    // node arrays, which are then grown (at least doubled) before the build
    // goes on from that level (the moment pass waits for a finished tree).
    int init_from = 0;
    for (;;) {
      TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
      LevelArgs A;
      A.in = pts_dev;
      A.pbuf0 = pbuf[0]; A.pbuf1 = pbuf[1];
      A.perm0 = perm2[0]; A.perm1 = perm2[1];
      A.pnode0 = pnode[0]; A.pnode1 = pnode[1];
      A.flag = flag; A.leftpos = leftpos; A.bcnt = bcnt;
      A.lo = t->lo; A.hi = t->hi; A.beg = t->beg; A.cnt = t->cnt; A.left = t->left; A.parent = t->parent;
      A.nleft = ns.nleft; A.arrive = ns.arrive; A.lp0 = ns.lp0; A.sloc = ns.sloc; A.leaves = t->leaves;
      A.lv = lv; A.ctl = ctl; A.bar = bar;
      A.wait = ctx->wait;
      A.n = n; A.d = d; A.dp = t->dp; A.leaf = t->leaf;
      A.cap = (int)std::min<size_t>(cap, INT32_MAX);
      A.init_from = init_from;
      A.max_levels = kMaxLevels;
      void* args[] = {&A};
      TRY(cudaLaunchCooperativeKernel((const void*)k_build_levels, dim3(ctx->build_grid), dim3(kBT), args, 0, s));
      ++*L;
      TRY(cudaEventRecord(t->tev[1], s));
      // the moment pass runs on the side stream after the level build; the
      // next call on the context overlaps it (readers wait on t->ready)
      TRY(cudaEventRecord(ctx->ev[4], s));
      TRY(cudaStreamWaitEvent(ctx->side, ctx->ev[4], 0));
      TRY(cudaEventRecord(t->tev[2], ctx->side));
      MomArgs M;
      M.pbuf0 = pbuf[0]; M.pbuf1 = pbuf[1];
      M.lo = t->lo; M.hi = t->hi; M.beg = t->beg; M.cnt = t->cnt; M.left = t->left; M.leaves = t->leaves;
      M.mom = t->mom; M.chi = t->chi; M.clo = t->clo; M.whalf = t->whalf; M.mnorm = t->mnorm; M.rad = t->rad;
      M.parent = t->parent; M.arrive = ns.arrive; M.ctl = ctl;
      M.n = n; M.d = d; M.dp = t->dp; M.pm = t->pm; M.P = t->P;
      switch (d) {
        case 1: TRY(launch_moments<1>(ctx, M, ctx->side)); break;
        case 2: TRY(launch_moments<2>(ctx, M, ctx->side)); break;
        case 3: TRY(launch_moments<3>(ctx, M, ctx->side)); break;
        case 4: TRY(launch_moments<4>(ctx, M, ctx->side)); break;
        case 5: TRY(launch_moments<5>(ctx, M, ctx->side)); break;
        default: TRY(launch_moments<0>(ctx, M, ctx->side)); break;
      }
      ++*L;
      TRY(cudaEventRecord(t->tev[3], ctx->side));
      TRY(cudaEventRecord(ctx->moments_done, ctx->side));
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
      // grow: a new arena and node scratch, the finished levels copied over
      // (once the moment pass, which found the tree unfinished, is done)
      TRY(cudaStreamSynchronize(ctx->side));
      const size_t nc = std::max(need + need / 2, cap * 2);
      const size_t nl = (size_t)h_ctl[3];
      dfgt_tree old = *t;
      DevBuf nsb;
      NodeScratch ns2;
      cudaError_t ce = alloc_tree(ctx, t, np, nc);
      if (ce == cudaSuccess) ce = nsb.ensure(NodeScratch::bytes(nc));
      if (ce == cudaSuccess) {
        ns2.carve(nsb.as<char>(), nc);
        ce = copy_d2d(t->lo, old.lo, keep * d * sizeof(float), s, ce);
        ce = copy_d2d(t->hi, old.hi, keep * d * sizeof(float), s, ce);
        ce = copy_d2d(t->beg, old.beg, keep * sizeof(int), s, ce);
        ce = copy_d2d(t->cnt, old.cnt, keep * sizeof(int), s, ce);
        ce = copy_d2d(t->left, old.left, keep * sizeof(int), s, ce);
        ce = copy_d2d(t->parent, old.parent, keep * sizeof(int), s, ce);
        ce = copy_d2d(t->leaves, old.leaves, nl * sizeof(int), s, ce);
        ce = copy_d2d(ns2.nleft, ns.nleft, keep * sizeof(int), s, ce);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(ns2.arrive, 0, keep * sizeof(int), s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      }
      if (old.arena != t->arena) {
        // the arena that is not kept goes back to the pool
        std::lock_guard<std::mutex> g(ctx->tpool->m);
        cudaFreeAsync(ce == cudaSuccess ? old.arena : t->arena, s);
        if (ce != cudaSuccess) *t = old;
      }
      if (ce != cudaSuccess) {
        nsb.release();
        ctx->err = std::string("dfgt_build: growing the node arrays: ") + cudaGetErrorString(ce);
        goto fail;
      }
      ctx->bnodes.release();
      ctx->bnodes = nsb;
      ns = ns2;
      cap = nc;
      init_from = (int)keep;
    }
    TRY(cudaEventRecord(t->ready, ctx->side));
    const int last = h_ctl[2];
    const int cur = h_ctl[1];
    TRY(copy_d2d(t->pts, pbuf[cur], np * t->dp * sizeof(float), s, cudaSuccess));
    TRY(copy_d2d(t->perm, perm2[cur], np * sizeof(int), s, cudaSuccess));
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
  rc = DFGT_OK;
fail:
  if (rc != DFGT_OK) {
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(ctx->side);
    free_tree(t);
  }
  return rc;
}

}  // namespace dfgt
