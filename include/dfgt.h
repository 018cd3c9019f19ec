/*
 * dfgt.h -- C ABI of the GB300 dual-tree fast Gauss transform library.
 *
 * The library computes Gaussian kernel sums (Eq. 5 of Lee, Gray & Moore,
 * "Dual-Tree Fast Gauss Transforms")
 *
 *     G(q_i) = sum_j exp(-||q_i - r_j||^2 / (2 h^2))
 *
 * for every query q_i, either exactly (brute force) or with a per-query
 * relative error bound |G~(q_i) - G(q_i)| <= eps * G(q_i) (Definition 1.2)
 * by the dual-tree traversal of Section 3.6.  All compute runs in CUDA
 * kernels on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Points are row-major float32 arrays [n][d], 1 <= d <= 32.
 *   - "_dev" pointers are device memory on the context's device and are
 *     owned by the caller; "_host" pointers are host memory owned by the
 *     caller.  The library never frees or keeps caller memory.
 *   - Trees and contexts are opaque and owned by the library; free them
 *     with dfgt_tree_destroy / dfgt_destroy.
 *   - Every call is enqueued on the context's stream and returns only
 *     after that work has finished and its status word has been read back.
 *     No call aborts, traps or throws; failures come back as a status and
 *     a message from dfgt_last_error.
 *   - Invalid arguments return DFGT_EINVAL before anything is launched.
 *   - One context serves one host thread at a time.
 */
#ifndef DFGT_H
#define DFGT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DFGT_OK = 0,
  DFGT_EINVAL = 1,        /* an argument is out of range; nothing was launched */
  DFGT_ENOMEM = 2,        /* a device or pinned-host allocation failed */
  DFGT_ECUDA = 3,         /* a CUDA runtime call failed (message in dfgt_last_error) */
  DFGT_ECAPACITY = 4,     /* a device work list overflowed its hard size limit */
  DFGT_ETIMEOUT = 5,      /* a bounded loop (tree levels, traversal rounds) ran out */
  DFGT_EUNSUPPORTED = 6   /* valid request this build does not implement */
} dfgt_status;

typedef struct dfgt_ctx dfgt_ctx;   /* device, stream, cached workspace */
typedef struct dfgt_tree dfgt_tree; /* permuted points, kd-tree nodes, raw moments */

/* Build and traversal options.  Zero-initialised means "defaults". */
typedef struct {
  int leaf_size;   /* leaf threshold of Algorithm 2 (BuildKdTree); 0 -> 128; max 256 */
  int p_max;       /* per-dimension expansion order limit; 0 -> the paper's table
                      (Section 3.6: 6 for D=2, 4 for D=3, 2 for D=4,5, 1 for D>=6;
                      8 for D=1); a smaller positive value lowers it */
  double eps_fp;   /* part of eps reserved for float32 rounding in exact sums;
                      0 -> chosen per sum: 1% of eps within [2e-5, 1e-4] for
                      d <= 5, half of eps within [2e-5, 5e-3] for d >= 6
                      (a sum takes the larger of its two trees' values);
                      must be < eps */
  long long base_block; /* a node pair that no summary can take is summed exactly,
                      without splitting further, once |Q| |R| <= base_block;
                      0 -> 4096, -1 -> only leaf pairs (as in DFGT) */
} dfgt_opts;

/* Work counters of one dfgt_sum call, summed over its bandwidths. */
typedef struct {
  long long pairs_visited;      /* node pairs classified */
  long long n_prune;            /* pairs summarised by the distance-bound prune */
  long long n_farfield;         /* pairs summarised by far-field evaluation (F) */
  long long n_local;            /* pairs summarised by direct local accumulation (D) */
  long long n_f2l;              /* pairs summarised by far-to-local translation (T) */
  long long n_base;             /* leaf pairs summed exactly (DFGTBase) */
  long long base_interactions;  /* sum over base pairs of |Q_leaf| * |R_leaf| */
  long long kernel_launches;    /* kernels this call launched */
  int rounds;                   /* level-synchronous traversal rounds */
  int list_flushes;             /* times an action list was drained before the traversal ended */
  double ms_traverse;           /* device time of the traversal rounds (with early list drains) */
  double ms_classify;           /* device time of the classification kernels of all rounds */
  double ms_actions;            /* device time of the final list drains */
  double ms_post;               /* device time of the downward pass and finalisation */
  double ms_base;               /* device time of every base-case (DFGTBase) launch */
  double ms_farfield;           /* device time of every far-field evaluation launch */
  double ms_local;              /* device time of every direct local accumulation launch */
  double ms_f2l;                /* device time of every far-to-local translation launch */
  long long base_expanded;      /* part of base_interactions summed in the expanded form
                                   (FMA pipe for D <= 5, tensor cores for D >= 6) */
  long long farfield_terms;     /* sum over far-field pairs of |Q| p^D (terms evaluated) */
  long long local_terms;        /* sum over direct local pairs of |R| p^D (terms accumulated) */
  long long f2l_terms;          /* sum over far-to-local pairs of p^{2D} (coefficient products) */
  long long log_queries;        /* dfgt_sum_log: (bandwidth, query) pairs summed in log space */
  double ms_log;                /* dfgt_sum_log: device time of the log-space pass */
  double ms_base_tc;            /* part of ms_base spent in the tensor-core exact sums (D >= 6) */
} dfgt_stats;

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t to run on (not owned), or NULL to create a private
 * non-blocking stream. */
dfgt_status dfgt_create(dfgt_ctx** out, int device, void* cuda_stream);

/* Set the capacity of the traversal's action lists (items per list) and
 * the initial capacity of its frontier (node pairs).  A list that could
 * overflow in the next round is drained first (its kernel runs early,
 * counted in dfgt_stats.list_flushes); the frontier grows to hold the
 * next round's child pairs (at most four per pair).  Larger lists trade memory for fewer, larger
 * launches.  Both must be >= 1. */
dfgt_status dfgt_set_capacity(dfgt_ctx* ctx, int64_t frontier_pairs, int64_t list_items);

/* Free a context and its cached workspace.  NULL is ignored. */
void dfgt_destroy(dfgt_ctx* ctx);

/* Number of CUDA kernels this context has launched since it was created
 * (tree builds, sums, brute force); -1 for a NULL context. */
long long dfgt_launch_count(const dfgt_ctx* ctx);

/* Test switch for the error path of the bounded device-side waits (no
 * counterpart in the paper).  The tree build and the traversal each run as
 * one cooperative launch whose blocks meet at grid barriers; every wait
 * there polls at most 2^25 times (about a second), then the block records a
 * timeout in the call's status word and returns, and the call returns
 * DFGT_ETIMEOUT.  With on = 1 every such barrier of this context waits for
 * one arrival more than the grid has and gives up after 4096 polls, so each
 * block leaves at its first barrier and dfgt_build / dfgt_sum return
 * DFGT_ETIMEOUT within milliseconds, with no kernel left running and the
 * context still usable.  on = 0 restores the normal waits.  Nothing traps or
 * faults; other values of `on` give DFGT_EINVAL. */
dfgt_status dfgt_test_wait_timeout(dfgt_ctx* ctx, int on);

/* Message of the last failure on this context ("" if none).  The string
 * belongs to the context and lives until the next call on it. */
const char* dfgt_last_error(const dfgt_ctx* ctx);

/* Build the mid-point kd-tree of Algorithm 2 (BuildKdTree, Section 2.1)
 * over n points (points_dev: float32 [n][d], device, caller-owned, not
 * modified) and the raw far-field moments of every node
 * (Eq. far_field_moments; leaves directly, internal nodes by the
 * far-to-far translation of Lemma 3.5).  The tree keeps its own permuted
 * copy of the points.  n >= 1, 1 <= d <= 32, finite coordinates. */
dfgt_status dfgt_build(dfgt_ctx* ctx, const float* points_dev, int64_t n, int d,
                       const dfgt_opts* opts, dfgt_tree** out);

/* Leave-one-out sums over one point set: for every point x_i (tree order
 * undone, caller's order) and bandwidth h_host[k],
 *   S_dev[k * n + i] = sum_{j != i} exp(-|x_i - x_j|^2 / 2h^2)
 * with |S~ - S| <= eps S (Definition 1.2 for the leave-one-out sum itself).
 * The dual-tree recursion runs with the query tree equal to the reference
 * tree; a node pair whose point ranges meet counts |R| - 1 other points in
 * its lower bound and error budget, is summarised only when R holds all of
 * Q (the summary's exact self term 1 is then taken off), and otherwise goes
 * to the exact sums, which leave the self interaction out.  Duplicate
 * points are other points.  n >= 2; otherwise as dfgt_sum. */
dfgt_status dfgt_sum_loo(dfgt_ctx* ctx, const dfgt_tree* tree, const double* h_host, int nh, double eps,
                         double* S_dev, dfgt_stats* stats);

/* Cross-validation scores of a bandwidth sweep over one point set (the
 * introduction's CV_LK and CV_LS, with the density estimate of Eq. 1 for
 * the Gaussian kernel, V_{D,h} = (2 pi h^2)^{D/2}).  `tree` holds the
 * reference set, which is also the query set; for each h_host[k]
 *   cv_lk[k] = (1/N) sum_j log( S_j / ((N-1) V_{D,h}) ),
 *   cv_ls[k] = (1/N) sum_j ( S*_j / ((N-1) V_{D,sqrt2 h}) - 2 S_j / ((N-1) V_{D,h}) ),
 * S_j the leave-one-out sum at h and S*_j at sqrt(2) h (the convolution
 * kernel K_h * K_h; the text's "bandwidth 2h" is read as variance 2h^2).
 * Runs dfgt_sum_loo over the 2 nh bandwidths {h, sqrt(2) h}, so every
 * leave-one-out sum has |S~_j - S_j| <= eps S_j, then reduces on the device
 * in float64.  lk_bound[k] and ls_bound[k] (may be NULL) bound
 * |score - exact score| from that guarantee: -log(1 - eps) and
 * (1/N) sum_j eps' (S~*_j / ((N-1) V*) + 2 S~_j / ((N-1) V)),
 * eps' = eps / (1 - eps); an estimate S~_j <= 0 (a point with no
 * neighbour above float32 underflow) gives a score of -inf and an infinite
 * lk bound.
 * Host outputs have nh entries; 1 <= nh <= 512; N >= 2. */
dfgt_status dfgt_cv_scores(dfgt_ctx* ctx, const dfgt_tree* tree, const double* h_host, int nh,
                           double eps, double* cv_lk_host, double* cv_ls_host,
                           double* lk_bound_host, double* ls_bound_host, dfgt_stats* stats);

/* Gradient of the leave-one-out likelihood score CV_LK (introduction) with
 * respect to log h and to every point, from exact sums (the adjoint of the
 * score's definition; no approximation).  With K_ij = exp(-|x_i-x_j|^2/2h^2)
 * and S_i = sum_{j != i} K_ij:
 *   cv[k]        = (1/N) sum_i log(S_i / ((N-1) V_{D,h})),
 *   dcv_dlogh[k] = (1/N) sum_i sum_{j != i} K_ij |x_i - x_j|^2 / (h^2 S_i) - D,
 *   dcv_dx[k][i] = -(1/(N h^2)) sum_{j != i} K_ij (x_i - x_j) (1/S_i + 1/S_j).
 * x_dev: float32 [n][d] points (device, caller-owned, row-major); they are
 * the query and the reference set.  h_host: nh bandwidths (host).
 * cv, dcv_dlogh: host arrays of nh; dcv_dx_dev: device float64
 * [nh][n][d], or NULL for the scalars only.  Two passes over all n^2 pairs
 * per bandwidth (kernel values in float32, sums in float64).
 * 2 <= n < 2^29, 1 <= d <= 32, 1 <= nh <= 512; a point with no neighbour
 * above float32 underflow (S_i = 0) makes cv = -inf and its gradient NaN. */
dfgt_status dfgt_cv_grad(dfgt_ctx* ctx, const float* x_dev, int64_t n, int d, const double* h_host, int nh,
                         double* cv, double* dcv_dlogh, double* dcv_dx_dev);

/* The boundary's gradient entry point: the same call, arguments and
 * results as dfgt_cv_grad (the leave-one-out likelihood score and its
 * gradients with respect to log h and to every point). */
dfgt_status dfgt_grad(dfgt_ctx* ctx, const float* x_dev, int64_t n, int d, const double* h_host, int nh,
                      double* cv, double* dcv_dlogh, double* dcv_dx_dev);

/* Choose the tree options that make a dual-tree sum of these points
 * fastest on this GPU.  No counterpart in the paper (its leaf size is
 * unstated, and its p_max table is an upper limit, Section 3.6): the leaf
 * size, the exact-sum block base_block and the expansion order limit trade
 * traversal work, series work and exact-sum work, and the best choice
 * depends on the data, the bandwidths and eps.  Builds a tree over
 * points_dev (float32 [n][d], device, caller-owned, not modified) for each
 * candidate (leaf_size 32, 64, 96, 128, 160, 192; base_block 2048, 4096,
 * 8192; p_max the paper's table value and one below it, or the caller's
 * best->p_max alone if it is > 0), runs dfgt_sum(tree, tree,
 * h_host[0..nh), eps) trials + 1 times and keeps the fastest of the last
 * `trials` runs (build and sum, CUDA events on the context's stream).
 * `best` is read for p_max and eps_fp (eps_fp is kept) and receives the
 * chosen options; best_ms (may be NULL) the time of one build and sum
 * with them.  1 <= trials <= 16.  Results of the trial sums are discarded;
 * every candidate keeps the guarantee of Definition 1.2.  Errors as for
 * dfgt_build and dfgt_sum. */
dfgt_status dfgt_autotune(dfgt_ctx* ctx, const float* points_dev, int64_t n, int d,
                          const double* h_host, int nh, double eps, int trials,
                          dfgt_opts* best, double* best_ms);

/* Free a tree.  NULL is ignored. */
void dfgt_tree_destroy(dfgt_tree* tree);

/* Approximate G(q_i) for every query of `qtree` against every reference
 * of `rtree` (qtree may equal rtree: the cross-validation setting of the
 * introduction) for each of the nh bandwidths h_host[0..nh), with the
 * relative error bound eps of Definition 1.2 (Theorem 3.3), by the
 * dual-tree traversal of Section 3.6 (DFGTMain).
 *   h_host : nh finite values > 0 (host); 1 <= nh <= 1024
 *   eps    : 0 < eps < 1, above the trees' float allowance eps_fp (with
 *            eps_fp = 0 that is a share of eps with a floor of 2e-5, so
 *            eps > 2e-5); else DFGT_EINVAL
 *   G_dev  : float64 [nh][nq] (device, caller-owned), written in the
 *            caller's original query order; unnormalised sums of Eq. 5
 *   stats  : optional work counters (host), may be NULL
 * The guarantee holds for every query whose exact sum is above ~1e-30
 * (float32 range of the exact leaf sums); dfgt_sum_log extends it to every
 * query. */
dfgt_status dfgt_sum(dfgt_ctx* ctx, const dfgt_tree* qtree, const dfgt_tree* rtree,
                     const double* h_host, int nh, double eps, double* G_dev,
                     dfgt_stats* stats);

/* dfgt_sum with log G beside G, so that the guarantee of Definition 1.2
 * holds for every query, including queries whose sum (Eq. 5) lies below
 * the float32 or even the float64 range (far from every reference, small
 * h, large D).  Runs dfgt_sum, then every (bandwidth, query) whose estimate
 * is below 1e-20 is summed again in log space: with x_j = |q - r_j|^2/2h^2
 * and the shift m = min_j x_j, log G = -m + log sum_j exp(-(x_j - m)),
 * from a depth-first walk of the reference tree with double-float squared
 * distances; nodes whose every point is exp(-T) below the nearest one,
 * T = log(|R| / (eps/4)) + 1, are skipped (at most eps/4 of G in all).
 *   G_dev    : float64 [nh][nq] as for dfgt_sum (underflows to 0 where G does)
 *   logG_dev : float64 [nh][nq] (device, caller-owned), caller order: log G~
 * Guarantee: |exp(logG~ - log G) - 1| <= eps for every query.
 * stats (may be NULL) also receives log_queries and ms_log.  Arguments and
 * errors as dfgt_sum; DFGT_ECAPACITY if the reference tree is too deep for
 * the walk's stack (not reachable with the build's 128-level limit). */
dfgt_status dfgt_sum_log(dfgt_ctx* ctx, const dfgt_tree* qtree, const dfgt_tree* rtree,
                         const double* h_host, int nh, double eps, double* G_dev, double* logG_dev,
                         dfgt_stats* stats);

/* Exact G(q_i) by the all-pairs sum of Algorithm 1 (NaiveKDE, without its
 * normalisation) for nh bandwidths; float32 distances and exponentials,
 * compensated accumulation.
 *   q_dev  : float32 [nq][d] device;  r_dev : float32 [nr][d] device
 *   h_host : nh values > 0 (host), 1 <= nh <= 1024
 *   G_dev  : float64 [nh][nq] device, caller-owned */
dfgt_status dfgt_sum_bruteforce(dfgt_ctx* ctx, const float* q_dev, int64_t nq,
                                const float* r_dev, int64_t nr, int d, const double* h_host,
                                int nh, double* G_dev);

/* End-to-end convenience call on HOST buffers: copies the points to the
 * device, builds the tree(s), runs dfgt_sum and copies G back.  When
 * q_host == r_host and nq == nr one tree serves both sides.
 *   q_host, r_host : float32 [n][d] host (pinned memory is fastest)
 *   G_host         : float64 [nh][nq] host, caller-owned */
dfgt_status dfgt_kde_host(dfgt_ctx* ctx, const float* q_host, int64_t nq, const float* r_host,
                          int64_t nr, int d, const double* h_host, int nh, double eps,
                          const dfgt_opts* opts, double* G_host, dfgt_stats* stats);

/* Exact sums as dfgt_sum_bruteforce, for callers that cannot allocate
 * device memory: code running while a CUDA graph is captured, hosts that
 * give the library a fixed memory budget and forbid allocations of its own,
 * and loops where an allocation's implicit synchronisation is not
 * acceptable.  The paper has no counterpart; this is a library service.
 *
 * No context is needed and nothing is allocated.  A query set large enough
 * to fill the GPU is summed in one pass straight into G_dev; a smaller one
 * splits the references into slices whose float64 partial sums live in a
 * 16 MiB static device array that every GPU loading the library reserves
 * until the process exits.  Limit of the split case: nh * nq <= 1,048,576
 * (partials of two slices must fit); larger split requests return
 * DFGT_ECAPACITY before anything is launched.
 *   q_dev, r_dev : float32 [n][d] on the current device (caller-owned,
 *                  contiguous rows)
 *   h_host       : nh finite bandwidths > 0 (host), 1 <= nh <= 1024
 *   G_dev        : float64 [nh][nq] on the current device (caller-owned)
 *   cuda_stream  : cudaStream_t to run on (NULL = the legacy default stream)
 * The call enqueues its kernels and returns; G_dev is complete once the
 * stream reaches that point.  All calls share the static array: calls whose
 * kernels overlap on the GPU (different streams, or several host threads)
 * race on it and corrupt each other's results; calls on one stream are
 * ordered and safe.  The first split call on a device looks up the array's
 * device address (cudaGetSymbolAddress, which may load the module) and
 * keeps it for the life of the process; make that first call before any
 * stream capture, and do not use this entry point after a device reset
 * (cudaDeviceReset), which leaves the kept address stale.  Errors:
 * DFGT_EINVAL for bad arguments, DFGT_ECAPACITY past the limit, DFGT_ECUDA
 * if a launch fails. */
dfgt_status dfgt_sum_bruteforce_static(const float* q_dev, int64_t nq, const float* r_dev,
                                       int64_t nr, int d, const double* h_host, int nh,
                                       double* G_dev, void* cuda_stream);

/* ---- introspection (used by the tests; not on the hot path) ---- */

typedef struct {
  int64_t n_points;
  int d;
  int n_nodes;     /* nodes are numbered level by level (breadth-first) */
  int n_leaves;
  int depth;       /* number of levels */
  int leaf_size;
  int p_max;       /* storage radix of the coefficient tables */
  int n_coeff;     /* p_max^d coefficients per node */
  double ms_levels;   /* device time of the build up to the end of its level build
                         (root set-up and the cooperative level launch) */
  double ms_moments;  /* device time of the moment pass (Eq. far_field_moments and
                         Lemma 3.5 translations; it runs on the context's side stream) */
} dfgt_tree_info;

/* Sizes of a tree and the device times of its build; waits for the build's
 * moment pass to finish. */
dfgt_status dfgt_tree_get_info(const dfgt_tree* tree, dfgt_tree_info* out);

/* Copy the tree to caller-owned HOST buffers; any pointer may be NULL.
 *   perm    int32  [n]          original index of the point at each position
 *   lo, hi  float32[n_nodes][d] tight bounding box of each node (Algorithm 2)
 *   begin, count int32 [n_nodes] the node's points are positions [begin, begin+count)
 *   left    int32  [n_nodes]    first child (the second is left+1), -1 for a leaf
 *   moments float64[n_nodes][n_coeff] raw moments m_alpha = sum_r (r-c)^alpha/alpha!
 *           about the box center c, multi-index alpha at position
 *           sum_d alpha[d] p_max^(d_count-1-d) (last dimension least significant);
 *           the h-scaled moments of Eq. far_field_moments are m_alpha (2h^2)^(-|alpha|/2).
 *   radius  float32[n_nodes]    radius of the node's points about the float box centre
 *           0.5f (lo + hi), rounded up (the ball that tightens the distance bounds for
 *           d >= 6). */
dfgt_status dfgt_tree_export(const dfgt_tree* tree, int32_t* perm, float* lo, float* hi,
                             int32_t* begin, int32_t* count, int32_t* left, double* moments,
                             float* radius);

/* Actions of Summarize / DFGTBase applied to explicit node pairs. */
enum {
  DFGT_ACT_PRUNE = 0,    /* |R|(K(d^l)+K(d^u))/2 to every query of Q */
  DFGT_ACT_FARFIELD = 1, /* EvaluateFarFieldExpansion of R at the queries of Q, order p */
  DFGT_ACT_LOCAL = 2,    /* AccumulateDirectLocalMoment of R into Q, order p */
  DFGT_ACT_F2L = 3,      /* TransFarToLocal of R's moments into Q, order p */
  DFGT_ACT_BASE = 4      /* DFGTBase: exact sum (both nodes must be leaves) */
};

/* Apply the listed actions for one bandwidth h and write, for every query
 * of qtree, the sum of their contributions after the downward pass
 * (TransLocalToLocal + EvaluateLocalExpansion, DFGTPost) into G_dev
 * (float64 [nq], caller order).  qnode/rnode/action/order are host arrays
 * of length n (order in 1..p_max, ignored for prune and base).  This runs
 * the same kernels as dfgt_sum on a caller-chosen pair list; it exists so
 * each operator can be checked against a reference.  The exact sums take
 * the trees' float allowance eps_fp (2e-5 where both leave it 0).  stats
 * (may be NULL) receives base_interactions and base_expanded of the listed
 * exact sums. */
dfgt_status dfgt_apply_pairs(dfgt_ctx* ctx, const dfgt_tree* qtree, const dfgt_tree* rtree,
                             const int32_t* qnode_host, const int32_t* rnode_host,
                             const int32_t* action_host, const int32_t* order_host, int n,
                             double h, double* G_dev, dfgt_stats* stats);

#ifdef __cplusplus
}
#endif

#endif /* DFGT_H */
