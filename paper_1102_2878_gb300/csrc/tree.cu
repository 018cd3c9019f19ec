// tree.cu -- device build of the mid-point kd-tree (Algorithm 2, BuildKdTree)
// and of the raw far-field moments of every node (Eq. far_field_moments at
// the leaves, the far-to-far translation of Lemma 3.5 upward).
//
// The build is level-synchronous: every level computes the tight bounding
// box of each of its nodes, splits the widest dimension at the box
// midpoint when the node holds more points than the leaf threshold, and
// stably partitions the points of every split node (x[sd] <= sc to the
// left) with one device-wide prefix sum.  Nodes are numbered level by
// level, so each level is a contiguous index range and the two children of
// a node are adjacent.  A split that would leave one side empty (all
// points equal along the widest side, or a midpoint that rounds onto the
// upper bound) turns the node into a leaf.
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

__global__ void k_pad_points(const float* __restrict__ in, int n, int d, int dp,
                             float* __restrict__ out, int* __restrict__ perm,
                             int* __restrict__ pnode, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool bad = false;
  for (int k = 0; k < dp; ++k) {
    float v = k < d ? in[(size_t)i * d + k] : 0.f;
    if (!isfinite(v)) bad = true;
    out[(size_t)i * dp + k] = v;
  }
  perm[i] = i;
  pnode[i] = 0;
  if (bad) atomicOr(status, kStNonFinite);
}

// The root: all points, an empty box to be filled by k_bbox; level 0 = [0, 1).
__global__ void k_init_root(int n, int d, int* beg, int* cnt, int* left, int* parent, float* lo, float* hi,
                            int* lv) {
  if (threadIdx.x == 0) {
    beg[0] = 0;
    cnt[0] = n;
    left[0] = -1;
    parent[0] = -1;
    lv[0] = 0;
    lv[1] = 1;
  }
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
}

// Tight bounding boxes of the nodes of the current level (min/max over each
// node's points).  Points are contiguous per node, so most blocks see one
// node and reduce in shared memory before one atomic per coordinate.
__global__ void __launch_bounds__(kT) k_bbox(const float* __restrict__ pts, int n, int d, int dp,
                                             const int* __restrict__ pnode, float* lo, float* hi) {
  __shared__ int s_nd;
  __shared__ float s_min[kT / 32], s_max[kT / 32];
  const int i = blockIdx.x * kT + threadIdx.x;
  const int nd = i < n ? pnode[i] : -1;
  if (threadIdx.x == 0) s_nd = nd;
  __syncthreads();
  const bool uniform = __syncthreads_and(nd == s_nd);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (uniform) {
    if (nd < 0) return;
    for (int k = 0; k < d; ++k) {
      float v = pts[(size_t)i * dp + k];
      float mn = v, mx = v;
      for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (lane == 0) { s_min[wid] = mn; s_max[wid] = mx; }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int w = 1; w < kT / 32; ++w) { mn = fminf(mn, s_min[w]); mx = fmaxf(mx, s_max[w]); }
        atomic_min_f(&lo[(size_t)nd * d + k], mn);
        atomic_max_f(&hi[(size_t)nd * d + k], mx);
      }
      __syncthreads();
    }
    return;
  }
  // every lane of the warp is still present here (no lane has returned)
  const unsigned peers = __match_any_sync(0xffffffffu, nd);
  if (nd < 0) return;
  const int leader = __ffs(peers) - 1;
  for (int k = 0; k < d; ++k) {
    float v = pts[(size_t)i * dp + k];
    if (peers == 0xffffffffu) {
      float mn = v, mx = v;
      for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (lane == leader) {
        atomic_min_f(&lo[(size_t)nd * d + k], mn);
        atomic_max_f(&hi[(size_t)nd * d + k], mx);
      }
    } else {
      atomic_min_f(&lo[(size_t)nd * d + k], v);
      atomic_max_f(&hi[(size_t)nd * d + k], v);
    }
  }
}

// Split rule of a node: it splits only if it holds more than `leaf` points
// and its box has positive extent, along its widest side sd at the box
// midpoint sc (Algorithm 2).
__device__ __forceinline__ bool split_rule(int j, int d, int leaf, const int* __restrict__ cnt,
                                           const float* __restrict__ lo, const float* __restrict__ hi,
                                           int& sd, float& sc) {
  sd = 0;
  float ext = hi[(size_t)j * d] - lo[(size_t)j * d];
  for (int k = 1; k < d; ++k) {
    const float x = hi[(size_t)j * d + k] - lo[(size_t)j * d + k];
    if (x > ext) { ext = x; sd = k; }
  }
  sc = 0.5f * (lo[(size_t)j * d + sd] + hi[(size_t)j * d + sd]);
  return cnt[j] > leaf && ext > 0.f;
}

__global__ void k_flag_left(const float* __restrict__ pts, int n, int dp, int d, int leaf,
                            const int* __restrict__ pnode, const int* __restrict__ cnt,
                            const float* __restrict__ lo, const float* __restrict__ hi,
                            int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nd = pnode[i];
  int f = 0;
  int sd;
  float sc;
  if (nd >= 0 && split_rule(nd, d, leaf, cnt, lo, hi, sd, sc)) f = pts[(size_t)i * dp + sd] <= sc ? 1 : 0;
  flag[i] = f;
}

// Level L occupies nodes [lv[3L], lv[3L+1]); lv[3L+2] is its number of
// splits.  Node kernels of a level run over `bound` >= its node count.
__global__ void k_node_finalize(const int* __restrict__ lv, int L, int bound, int d, int leaf,
                                const int* __restrict__ beg, const int* __restrict__ cnt,
                                const float* __restrict__ lo, const float* __restrict__ hi,
                                const int* __restrict__ leftpos, int* __restrict__ split,
                                int* __restrict__ nleft) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= bound) return;
  const int a = lv[3 * L], e = lv[3 * L + 1];
  const int j = a + t;
  if (j >= e) {
    split[t] = 0;
    nleft[t] = 0;
    return;
  }
  int sd;
  float sc;
  const bool want = split_rule(j, d, leaf, cnt, lo, hi, sd, sc);
  const int b = beg[j], c = cnt[j];
  const int nl = leftpos[b + c] - leftpos[b];
  split[t] = (want && nl > 0 && nl < c) ? 1 : 0;
  nleft[t] = nl;
}

// Children of the level's split nodes, numbered level by level; also
// writes the next level's range.  The caller reserves room for every node
// the level can create; a request beyond `cap` is refused and flagged.
__global__ void k_make_children(int* __restrict__ lv, int L, int bound, int d, int cap,
                                const int* __restrict__ split, const int* __restrict__ soff,
                                const int* __restrict__ nleft, int* beg, int* cnt, int* left,
                                int* parent, float* lo, float* hi, int* __restrict__ status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = lv[3 * L], e = lv[3 * L + 1];
  const int total = soff[bound];
  const bool fits = (long long)e + 2LL * total <= cap;
  if (t == 0) {
    lv[3 * L + 2] = fits ? total : 0;
    lv[3 * (L + 1)] = e;
    lv[3 * (L + 1) + 1] = fits ? e + 2 * total : e;
    if (!fits) atomicOr(status, kStOverflow);
  }
  if (t >= bound) return;
  const int j = a + t;
  if (j >= e) return;
  if (!fits || !split[t]) {
    left[j] = -1;
    return;
  }
  const int c0 = e + 2 * soff[t];
  const int nl = nleft[t];
  left[j] = c0;
  beg[c0] = beg[j];
  cnt[c0] = nl;
  beg[c0 + 1] = beg[j] + nl;
  cnt[c0 + 1] = cnt[j] - nl;
  parent[c0] = parent[c0 + 1] = j;
  left[c0] = left[c0 + 1] = -1;
  for (int k = 0; k < d; ++k) {
    lo[(size_t)c0 * d + k] = lo[(size_t)(c0 + 1) * d + k] = INFINITY;
    hi[(size_t)c0 * d + k] = hi[(size_t)(c0 + 1) * d + k] = -INFINITY;
  }
}

__global__ void k_scatter(int n, int dp, const int* __restrict__ lv, int L, const float* __restrict__ pin,
                          const int* __restrict__ perm_in, const int* __restrict__ pnode_in,
                          const int* __restrict__ flag, const int* __restrict__ leftpos,
                          const int* __restrict__ beg, const int* __restrict__ left,
                          const int* __restrict__ nleft, float* __restrict__ pout,
                          int* __restrict__ perm_out, int* __restrict__ pnode_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = lv[3 * L];
  const int nd = pnode_in[i];
  int dst = i, child = -1;
  if (nd >= 0 && left[nd] >= 0) {
    const int b0 = beg[nd];
    const int lrank = leftpos[i] - leftpos[b0];
    if (flag[i]) {
      dst = b0 + lrank;
      child = left[nd];
    } else {
      dst = b0 + nleft[nd - a] + (i - b0 - lrank);
      child = left[nd] + 1;
    }
  }
  for (int k = 0; k < dp; ++k) pout[(size_t)dst * dp + k] = pin[(size_t)i * dp + k];
  perm_out[dst] = perm_in[i];
  pnode_out[dst] = child;
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
  int *beg, *cnt, *left, *parent;
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
  }
  void copy_to(float* lo2, float* hi2, int* beg2, int* cnt2, int* left2, int* parent2, size_t keep,
               int d, cudaStream_t s, cudaError_t* e) const {
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (*e == cudaSuccess) *e = cudaMemcpyAsync(lo2, lo, keep * d * sizeof(float), k, s);
    if (*e == cudaSuccess) *e = cudaMemcpyAsync(hi2, hi, keep * d * sizeof(float), k, s);
    if (*e == cudaSuccess) *e = cudaMemcpyAsync(beg2, beg, keep * sizeof(int), k, s);
    if (*e == cudaSuccess) *e = cudaMemcpyAsync(cnt2, cnt, keep * sizeof(int), k, s);
    if (*e == cudaSuccess) *e = cudaMemcpyAsync(left2, left, keep * sizeof(int), k, s);
    if (*e == cudaSuccess) *e = cudaMemcpyAsync(parent2, parent, keep * sizeof(int), k, s);
  }
};

// Grow the context's node buffer to `cap` nodes keeping the first `keep`.
cudaError_t grow_nodes(DevBuf& buf, NodeArrays& na, size_t keep, size_t cap, int d, cudaStream_t s) {
  DevBuf nb;
  cudaError_t e = nb.ensure(NodeArrays::bytes(cap, d));
  if (e != cudaSuccess) return e;
  Carver c{nb.as<char>()};
  NodeArrays nn;
  nn.carve(c, cap, d);
  na.copy_to(nn.lo, nn.hi, nn.beg, nn.cnt, nn.left, nn.parent, keep, d, s, &e);
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
  // ids, flags, prefix sums, per-level node temporaries, the level table
  float* pbuf[2];
  int* perm2[2];
  int* pnode[2];
  int *flag, *leftpos, *split, *soff, *nleft, *status, *lv;
  NodeArrays na;
  size_t cap = 0;
  int cur = 0, level = 0, last = -1;
  int h_status = 0;
  dfgt_status rc = DFGT_ECUDA;
  std::vector<int> lvh;

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
    leftpos = cv.take<int>(np + 1);
    split = cv.take<int>(np + 1);
    soff = cv.take<int>(np + 2);
    nleft = cv.take<int>(np + 1);
    status = cv.take<int>(1);
    lv = cv.take<int>(3 * (kMaxLevels + 2));
    if (pass == 0) {
      TRY(ctx->bscratch.ensure(cv.off));
      cv.base = ctx->bscratch.as<char>();
    }
  }
  TRY(cudaMemsetAsync(status, 0, sizeof(int), s));

  cap = std::max<size_t>(64, 4 * np / std::max(1, t->leaf) + 16);
  {
    TRY(ctx->bnodes.ensure(NodeArrays::bytes(cap, d)));
    // use all the room the buffer has
    const size_t fit = (ctx->bnodes.bytes - 6 * 256) / (8 * (size_t)d + 16);
    if (fit > cap && NodeArrays::bytes(fit, d) <= ctx->bnodes.bytes) cap = fit;
    Carver c{ctx->bnodes.as<char>()};
    na.carve(c, cap, d);
  }

  k_pad_points<<<(n + kT - 1) / kT, kT, 0, s>>>(pts_dev, n, d, t->dp, pbuf[0], perm2[0], pnode[0], status);
  k_init_root<<<1, 32, 0, s>>>(n, d, na.beg, na.cnt, na.left, na.parent, na.lo, na.hi, lv);
  *L += 2;
  TRY(cudaGetLastError());

  {
    // Levels run in batches between host synchronisations.  A node splits
    // only if it holds more than `leaf` points, so a level has at most
    // 2 floor(n / (leaf + 1)) nodes below the root and at most twice the
    // nodes of the level above: node kernels run over that bound and the
    // node arrays hold room for every node a batch can create.  The level
    // table records each level's range and split count; a level without
    // splits ends the tree (levels enqueued after it are empty and leave the
    // points in place).
    const long long max_level_nodes = std::max<long long>(1, 2LL * (n / (t->leaf + 1)));
    size_t known_e = 1;
    long long known_nl = 1;
    int batch = std::max(8, ctx->last_depth + 1);
    const int gp = (n + kT - 1) / kT;
    while (last < 0) {
      if (level >= kMaxLevels) {
        ctx->err = "dfgt_build: more than 128 tree levels";
        rc = DFGT_ETIMEOUT;
        goto fail;
      }
      const int nb = std::min(batch, kMaxLevels - level);
      std::vector<long long> bnd(nb + 1);
      bnd[0] = known_nl;
      size_t need = known_e;
      for (int k = 1; k <= nb; ++k) {
        bnd[k] = std::min(2 * bnd[k - 1], max_level_nodes);
        need += (size_t)bnd[k];
      }
      if (need > cap) {
        const size_t nc = std::max(need, cap * 2);
        TRY(grow_nodes(ctx->bnodes, na, known_e, nc, d, s));
        cap = nc;
      }
      for (int k = 0; k < nb; ++k) {
        const int Lk = level + k;
        const int bk = (int)std::max<long long>(1, bnd[k]);
        const int gn = (bk + kT - 1) / kT;
        k_bbox<<<gp, kT, 0, s>>>(pbuf[cur], n, d, t->dp, pnode[cur], na.lo, na.hi);
        k_flag_left<<<gp, kT, 0, s>>>(pbuf[cur], n, t->dp, d, t->leaf, pnode[cur], na.cnt, na.lo, na.hi, flag);
        *L += 2;
        TRY(cudaGetLastError());
        TRY(scan_exclusive(flag, leftpos, n, ctx->scan_tmp, s, L));
        k_node_finalize<<<gn, kT, 0, s>>>(lv, Lk, bk, d, t->leaf, na.beg, na.cnt, na.lo, na.hi, leftpos,
                                          split, nleft);
        ++*L;
        TRY(cudaGetLastError());
        TRY(scan_exclusive(split, soff, bk, ctx->scan_tmp, s, L));
        k_make_children<<<gn, kT, 0, s>>>(lv, Lk, bk, d, (int)std::min<size_t>(cap, INT32_MAX), split, soff,
                                          nleft, na.beg, na.cnt, na.left, na.parent, na.lo, na.hi, status);
        k_scatter<<<gp, kT, 0, s>>>(n, t->dp, lv, Lk, pbuf[cur], perm2[cur], pnode[cur], flag, leftpos,
                                    na.beg, na.left, nleft, pbuf[cur ^ 1], perm2[cur ^ 1], pnode[cur ^ 1]);
        *L += 2;
        TRY(cudaGetLastError());
        cur ^= 1;
      }
      lvh.resize(3 * (level + nb + 1));
      TRY(cudaMemcpyAsync(lvh.data(), lv, lvh.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(cudaStreamSynchronize(s));
      if (h_status & kStNonFinite) {
        ctx->err = "dfgt_build: non-finite coordinate";
        rc = DFGT_EINVAL;
        goto fail;
      }
      if (h_status & kStOverflow) {
        ctx->err = "dfgt_build: node capacity bound violated (internal error)";
        rc = DFGT_ECAPACITY;
        goto fail;
      }
      for (int k = 0; k < nb && last < 0; ++k)
        if (lvh[3 * (level + k) + 2] == 0) last = level + k;
      level += nb;
      if (last < 0) {
        known_e = (size_t)lvh[3 * level + 1];
        known_nl = (long long)lvh[3 * level + 1] - lvh[3 * level];
        batch = 8;
      }
    }
    t->lvl_off.assign(1, 0);
    for (int Lk = 0; Lk <= last; ++Lk) t->lvl_off.push_back(lvh[3 * Lk + 1]);
    ctx->last_depth = last + 1;
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
    cudaError_t ce = cudaMemcpyAsync(t->pts, pbuf[cur], np * t->dp * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t->perm, perm2[cur], np * sizeof(int), cudaMemcpyDeviceToDevice, s);
    na.copy_to(t->lo, t->hi, t->beg, t->cnt, t->left, t->parent, nn, d, s, &ce);
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
  {
    // the leaf list, in node order, from the level structure
    std::vector<int> left_h(t->nn);
    TRY(cudaMemcpyAsync(left_h.data(), t->left, t->nn * sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    std::vector<int> leaves_h;
    for (int j = 0; j < t->nn; ++j)
      if (left_h[j] < 0) leaves_h.push_back(j);
    t->nleaves = (int)leaves_h.size();
    TRY(cudaMemcpyAsync(t->leaves, leaves_h.data(), leaves_h.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    TRY(cudaStreamSynchronize(s));
  }
  rc = DFGT_OK;
fail:
  if (rc != DFGT_OK) {
    cudaStreamSynchronize(s);
    free_tree(t);
  }
  return rc;
}

}  // namespace dfgt
