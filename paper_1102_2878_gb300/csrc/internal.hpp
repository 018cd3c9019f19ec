// internal.hpp -- host-side structures of the DFGT library (not part of the ABI).
#pragma once

#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "dfgt.h"

// Grow-only device buffer.  Reallocation happens only between calls (the
// owning call has synchronised its stream), so old contents are dropped.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t want = need + need / 4 + 256;
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) bytes = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// Carves 256-byte aligned sub-arrays out of one allocation; with a null
// base it only adds up the bytes a layout needs.
struct Carver {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Stream-ordered memory pool that tree arenas come from.  Shared by the
// context that creates it and every tree built on that context, so it
// lives until the last of them is gone; freed arenas stay cached in the
// pool for the next build instead of going back to the driver.
struct TreePool {
  cudaMemPool_t pool = nullptr;
  std::mutex m;
  cudaStream_t stream = nullptr;  // the owning context's stream while it lives
  ~TreePool() {
    if (pool) cudaMemPoolDestroy(pool);
  }
};

// Counters read back after each traversal round (one pinned copy).
struct RoundCounters {
  int n_next;          // pairs written to the next frontier
  int status;          // kSt* bits
  int n_far, n_loc, n_f2l, n_base;   // cumulative list lengths
  unsigned long long n_prune;        // cumulative prune count
  unsigned long long base_inter;     // cumulative sum |Q||R| over base pairs
  unsigned long long base_exp;       // base interactions summed in the expanded form
  unsigned long long far_terms;      // sum |Q| p^D over far-field actions
  unsigned long long loc_terms;      // sum |R| p^D over direct local actions
  unsigned long long f2l_terms;      // sum p^{2D} over far-to-local actions
};

constexpr int kCtxEvents = 18;  // [16], [17]: around the tensor-core exact sums

struct dfgt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;          // the moment pass of a build runs here
  cudaEvent_t moments_done = nullptr;   // the last moment pass issued on `side`
  std::string err;
  long long launches = 0;
  // cached workspace
  DevBuf scan_tmp;
  DevBuf counters;       // RoundCounters on the device
  DevBuf hvals;          // bandwidths, then 1/(2h^2)
  DevBuf kus;            // per frontier pair: K(d^u) lower and K(d^l) upper bounds, box sides
  DevBuf frontier[2];    // Pair
  DevBuf grp_cnt, grp_off, grp_r;  // base-case grouping scratch
  DevBuf tc_plan;        // tensor-core plan of the exact sums (D >= 6)
  DevBuf list_far, list_loc, list_f2l, list_base;  // Action / Pair
  DevBuf node_state;     // u64 inherited/decided/incr/lbsum
  DevBuf lmom;           // double local moments [nh][nn][P]
  DevBuf pused;          // int [nh][nn]
  DevBuf gacc;           // double [nh][nq]
  DevBuf io_q, io_r, io_g;  // dfgt_kde_host staging
  DevBuf bf_partials;       // brute-force slice partials
  DevBuf cv_buf;            // cross-validation normalisers, partials and scores
  DevBuf grad_buf;          // exact CV gradient sums (S, A, P, Y, partials)
  DevBuf log_items;         // (query, bandwidth chunk) items of the log-space pass
  DevBuf log_ctr;           // item count, flagged count and status of the log-space pass
  DevBuf bscratch;          // tree-build per-point scratch
  DevBuf bnodes;            // tree-build per-node scratch (left counts, prefixes, split ranks)
  std::shared_ptr<TreePool> tpool;
  int sms = 0;                // SMs of the device (0: not yet queried)
  int build_grid = 0;         // blocks of the cooperative level build (0: not yet chosen)
  int trav_grid[6] = {};      // blocks of the cooperative traversal per dimension template
  DevBuf trav_ctl;            // TravControl and the traversal's grid-barrier counter
  int mom_grid[6] = {};       // blocks of the cooperative moment pass per dimension (0: D >= 6)
  dfgt::BarrierCfg wait;      // grid-barrier waits of the cooperative launches
  size_t cap_frontier = 1 << 20;
  size_t cap_lists = 1 << 22;
  RoundCounters* h_counters = nullptr;  // pinned
  cudaEvent_t ev[kCtxEvents] = {};
};

struct dfgt_tree {
  int device = 0;
  cudaEvent_t ready = nullptr;  // moments and float node data written (recorded on the building context's side stream)
  cudaEvent_t tev[4] = {};      // build start, after the (last) level build; around the (last) moment pass
  int64_t n = 0;
  int d = 0, dp = 0, leaf = 32, pm = 1, P = 1, p_limit = 1;
  long long base_block = 0;
  double eps_fp = 2e-5;
  int nn = 0, nleaves = 0, depth = 0;
  std::vector<int> lvl_off;  // nodes of level k are [lvl_off[k], lvl_off[k+1])
  std::shared_ptr<TreePool> tpool;
  void* arena = nullptr;     // one pool allocation holding every array below
  float* pts = nullptr;
  int* perm = nullptr;
  float* lo = nullptr;
  float* hi = nullptr;
  int* beg = nullptr;
  int* cnt = nullptr;
  int* left = nullptr;
  int* parent = nullptr;
  int* leaves = nullptr;      // [nleaves] leaf node ids
  double* mom = nullptr;
  float* chi = nullptr;
  float* clo = nullptr;
  float* whalf = nullptr;
  float* mnorm = nullptr;
  float* rad = nullptr;       // radius of each node's points about its box centre
  dfgt::TreeView view() const {
    dfgt::TreeView v;
    v.pts = pts; v.perm = perm; v.lo = lo; v.hi = hi; v.beg = beg; v.cnt = cnt;
    v.left = left; v.parent = parent; v.mom = mom;
    v.chi = chi; v.clo = clo; v.whalf = whalf; v.mnorm = mnorm; v.rad = rad;
    v.n = (int)n; v.d = d; v.dp = dp; v.nn = nn; v.pm = pm; v.P = P;
    return v;
  }
};

namespace dfgt {

// scan.cu: exclusive prefix sum of n int32 values into out[0..n].
cudaError_t scan_exclusive(const int* in, int* out, int n, DevBuf& tmp, cudaStream_t s,
                           long long* launches);
// The same with 64-bit sums: out[0..n] of int64.
cudaError_t scan_exclusive64(const int* in, long long* out, int n, DevBuf& tmp, cudaStream_t s,
                             long long* launches);

// bruteforce.cu
// Slices the references are split into for nq queries (1 = no split).
int bruteforce_slices(int nq, int nr);
// With slices > 1, `partials` must hold slices * nh * nq doubles.
cudaError_t launch_bruteforce_split(const float* q, int nq, const float* r, int nr, int d,
                                    const double* h_host, int nh, double* G, int slices,
                                    double* partials, cudaStream_t s, long long* launches);
cudaError_t launch_bruteforce(const float* q, int nq, const float* r, int nr, int d,
                              const double* h_host, int nh, double* G, DevBuf& scratch,
                              cudaStream_t s, long long* launches);

// logsum.cu: log G (and G) of every (bandwidth, query) whose estimate in G
// (float64 [nh][nq], caller order) is below `flag`, by a depth-first walk
// of the reference tree with double-float distances and a per-query shift;
// log of the estimate elsewhere.  counters: one int (item count);
// n_flagged: listed (bandwidth, query) pairs; status: kSt* bits.
cudaError_t launch_log_pass(const TreeView& Q, const TreeView& R, const double* h_dev, int nh, double eps,
                            double flag, double* G, double* logG, DevBuf& items_buf, int* counters,
                            unsigned long long* n_flagged, int* status, cudaStream_t s, long long* launches,
                            int* n_items_host);

// cv.cu: cross-validation scores from the sums G [2 nh][n] at h and sqrt(2) h;
// part holds nh * nblk * 4 doubles, out nh * 4 (CV_LK, bound, CV_LS, bound).
cudaError_t launch_cv_scores(const double* G, int n, int nh, const double* norm, double eps, double* part,
                             int nblk, double* out, cudaStream_t s, long long* launches);

// cvgrad.cu: CV_LK, dCV/dlog h and dCV/dx at one bandwidth from exact sums.
// S, A: n doubles; P, Y: n*d doubles; part: 2*ceil(n/256) doubles; out[2] =
// {sum_i log S_i, sum_i A_i/(h^2 S_i)}; dx ([n][d], nullable) the point gradients.
cudaError_t launch_cv_grad(const float* X, int n, int d, double h, double* S, double* P, double* A, double* Y,
                           double* part, double* out, double* dx, cudaStream_t s, long long* launches);

// tree.cu: build the tree (points, nodes, raw moments) on ctx's stream.
dfgt_status build_tree(dfgt_ctx* ctx, const float* pts_dev, int64_t n, int d,
                       const dfgt_opts* opts, dfgt_tree* t);
void free_tree(dfgt_tree* t);

// traverse.cu / actions.cu launchers
struct TravBuffers {
  u64* inherited;   // [nh][nnQ]
  u64* decided;
  u64* incr;
  u64* lbsum;
  double* L;        // [nh][nnQ][P]
  int* pused;       // [nh][nnQ]
  double* gacc;     // [nh][nq] (permuted order)
  const double* h;  // [nh]
  const float* inv2h2_dn;  // [nh] 1/(2h^2) rounded down
  const float* inv2h2_up;  // [nh] 1/(2h^2) rounded up
  const float* inv_2h_up;  // [nh] 1/(2h) rounded up
  const float* c2;       // [nh] -log2(e)/(2h^2) as float, the exp2 scale of exact sums
  const float* sf;       // [nh] 1/sqrt(2h^2) as float, the expansion scale
  unsigned long long* base_exp;  // device counter of expanded-form base interactions
  int* status;           // device status word of the call (kSt* bits)
  float tau_scale_dn;    // eps_eff / (fix_scale |R_total|) as float, rounded down
  float* ku;        // [frontier] lower bound on K(d^u) of each pending pair
  float* kl;        // [frontier] upper bound on K(d^l), and the two boxes'
  float* sq;        //   largest sides, from the fold phase's box geometry,
  float* sr;        //   reused by the classification of the same pair
  int nh;
  double eps_eff;   // eps minus the float allowance for exact sums
  float exp_err;    // exponent error the expanded form of exact sums may take (eps_fp / 4)
  double fix_scale; // 2^62 / |R|
  double inv_fix;   // 1 / fix_scale
  float fix_scale_dn;  // fix_scale rounded down
  double inv_nr;    // 1 / |R|
  int p_limit;
  long long base_block;  // exact sum without recursing when |Q||R| <= this
  int sms;               // SMs of the device (sizes the balanced launches)
  int loo;               // leave-one-out sums: Q and R are one tree, each query's own term is left out
};

// State of the device-driven traversal between launches (device memory).
struct TravControl {
  int nF;              // pairs in the current frontier
  int cur;             // which frontier buffer holds them
  int rounds;          // rounds done
  int stop;            // why the last launch returned (kTrav*; -1 while running)
  long long visited;   // pairs classified so far
};
enum : int { kTravDone = 0, kTravRoom = 1, kTravRounds = 2, kTravOverflow = 3 };

cudaError_t launch_traverse(const TreeView& Q, const TreeView& R, const TravBuffers& b, Pair* F0, Pair* F1,
                            int cap_front, Action* far, Action* loc, Action* f2l, Pair* base, int cap_lists,
                            RoundCounters* ctr, TravControl* tc, unsigned* bar, const BarrierCfg& wait,
                            int max_rounds, int* grid, cudaStream_t s);
cudaError_t launch_init_frontier(Pair* F, int nh, cudaStream_t s);

// Scratch of the base-case grouping (counting sort by bandwidth and query node).
struct BaseScratch {
  DevBuf* cnt;
  DevBuf* off;
  DevBuf* rsorted;
  DevBuf* scan_tmp;
  DevBuf* plan;         // D >= 6: the tensor-core plan (items and per-entry flags)
  cudaEvent_t tc0 = nullptr, tc1 = nullptr;  // recorded around the tensor-core exact sums (D >= 6) if set
};
cudaError_t launch_base(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                        const Pair* list, int n, BaseScratch& sc, cudaStream_t s, long long* launches);
// base_tc.cu: the tensor-core runs of a sorted base list (D >= 6): the plan
// (which runs take the tensor form; tcflag[i] = 1 for their entries) and
// their sums.
// cnt[key] entries of key (bandwidth, query node) end at end[key] in the sorted list.
cudaError_t launch_tc_plan(const TreeView& Q, const TreeView& R, const TravBuffers& b, const int* rsorted,
                           const int* cnt, const int* end, int nkeys, int n, DevBuf& plan,
                           const unsigned char** tcflag, cudaStream_t s, long long* launches);
cudaError_t launch_tc_sums(const TreeView& Q, const TreeView& R, const TravBuffers& b, const int* rsorted, int n,
                           DevBuf& plan, cudaStream_t s, long long* launches);
cudaError_t launch_farfield(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                            const Action* list, int n, BaseScratch& sc, cudaStream_t s, long long* launches);
cudaError_t launch_local(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                         const Action* list, int n, BaseScratch& sc, cudaStream_t s,
                         long long* launches);
cudaError_t launch_f2l(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                       const Action* list, int n, cudaStream_t s);
cudaError_t launch_prune_apply(const TreeView& Q, const TreeView& R, const TravBuffers& b,
                               const Pair* list, int n, cudaStream_t s);
cudaError_t launch_post(const TreeView& Q, const int* leaves, int nleaves, const TravBuffers& b,
                        double* G, cudaStream_t s);

}  // namespace dfgt
