// api.cu -- the extern "C" entry points declared in include/dfgt.h and the
// host orchestration of one dual-tree sum (DFGTMain of Section 3.6):
// initialise the per-node state (DFGTInitQ), run traversal rounds until the
// frontier is empty, run the listed summaries and base cases, translate the
// local moments down the query tree and finalise (DFGTPost).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "internal.hpp"

using namespace dfgt;

namespace {

dfgt_status fail(dfgt_ctx* ctx, dfgt_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t _e = (x);                                                              \
    if (_e != cudaSuccess)                                                             \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? DFGT_ENOMEM : DFGT_ECUDA,     \
                  std::string(#x) + ": " + cudaGetErrorString(_e));                    \
  } while (0)

constexpr size_t kHardCap = size_t(1) << 28;  // entries per work list

bool bad_h(const double* h, int nh) {
  if (!h || nh < 1 || nh > 1024) return true;
  for (int i = 0; i < nh; ++i)
    if (!(h[i] > 0.0) || !std::isfinite(h[i])) return true;
  return false;
}

// DFGTPost: local expansions shifted to the leaves, read out and added to
// the exact and far-field parts, into G_dev (one fused kernel).
// Grow a buffer to `bytes`, keeping its first `keep` bytes.
cudaError_t grow_keep(DevBuf& buf, size_t bytes, size_t keep, cudaStream_t s) {
  if (bytes <= buf.bytes) return cudaSuccess;
  DevBuf nb;
  cudaError_t e = nb.ensure(bytes);
  if (e == cudaSuccess && keep) e = cudaMemcpyAsync(nb.p, buf.p, keep, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    nb.release();
    return e;
  }
  buf.release();
  buf = nb;
  return cudaSuccess;
}

// The stream waits until the tree's moment pass has run.
cudaError_t wait_ready(cudaStream_t s, const dfgt_tree* t) {
  return t->ready ? cudaStreamWaitEvent(s, t->ready, 0) : cudaSuccess;
}

dfgt_status post(dfgt_ctx* ctx, const dfgt_tree* qt, const TravBuffers& b, double* G_dev,
                 dfgt_stats* st) {
  cudaStream_t s = ctx->stream;
  const TreeView Q = qt->view();
  CK(wait_ready(s, qt));
  CK(launch_post(Q, qt->leaves, qt->nleaves, b, G_dev, s));
  ++ctx->launches;
  CK(cudaMemcpyAsync(ctx->h_counters, ctx->counters.p, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev[3], s));
  CK(cudaStreamSynchronize(s));
  if (st) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
    st->ms_post = ms;
  }
  return DFGT_OK;
}

// Part of eps reserved for float32 rounding in exact sums: the larger of
// the trees' eps_fp, or, where both leave it 0, 1% of eps within
// [2e-5, 1e-4] for D <= 5, half of eps within [2e-5, 5e-3] for D >= 6
// (where p_max = 1 leaves most of the work to exact sums, whose tensor
// form needs the room, and little but the prune to the expansions that
// eps - eps_fp budgets: at D = 16 and 32 half of eps gave the prune 1%
// fewer pairs than a fifth and moved two fifths to a half of the
// direct-form exact-sum interactions to the tensor form).
double float_allowance(const dfgt_tree* a, const dfgt_tree* b, double eps) {
  const double v = std::max(a->eps_fp, b->eps_fp);
  if (v > 0.0) return v;
  return a->d >= 6 ? std::min(5e-3, std::max(2e-5, 0.5 * eps)) : std::min(1e-4, std::max(2e-5, 0.01 * eps));
}

// Zeroed per-call state; returns the traversal buffers.
dfgt_status setup_state(dfgt_ctx* ctx, const dfgt_tree* qt, const dfgt_tree* rt, const double* h_host, int nh,
                        double eps_eff, double eps_fp, TravBuffers* b, bool loo = false) {
  cudaStream_t s = ctx->stream;
  const size_t nodes = (size_t)nh * qt->nn;
  CK(ctx->hvals.ensure(4 * (size_t)nh * sizeof(double)));
  CK(ctx->node_state.ensure(4 * nodes * sizeof(u64)));
  CK(ctx->lmom.ensure(nodes * qt->P * sizeof(double)));
  CK(ctx->pused.ensure(nodes * sizeof(int)));
  CK(ctx->gacc.ensure((size_t)nh * qt->n * sizeof(double)));
  CK(ctx->counters.ensure(sizeof(RoundCounters)));
  {
    // layout: h (double) | five float arrays inv_dn, inv_up, i2h_up, c2, sf
    std::vector<double> hv(4 * (size_t)nh);
    float* fl = reinterpret_cast<float*>(hv.data() + (size_t)nh);
    float* inv_dn = fl;
    float* inv_up = fl + nh;
    float* i2h_up = fl + 2 * (size_t)nh;
    float* c2 = fl + 3 * (size_t)nh;
    float* sfl = fl + 4 * (size_t)nh;
    for (int i = 0; i < nh; ++i) {
      hv[i] = h_host[i];
      const double inv = 1.0 / (2.0 * h_host[i] * h_host[i]);
      inv_dn[i] = std::nextafter((float)inv, 0.f);
      inv_up[i] = std::nextafter((float)inv, INFINITY);
      i2h_up[i] = std::nextafter((float)(1.0 / (2.0 * h_host[i])), INFINITY);
      c2[i] = (float)(-kLog2e * inv);
      sfl[i] = (float)(1.0 / std::sqrt(2.0 * h_host[i] * h_host[i]));
    }
    CK(cudaMemcpyAsync(ctx->hvals.p, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // hv is a stack buffer
  }
  CK(cudaMemsetAsync(ctx->node_state.p, 0, 4 * nodes * sizeof(u64), s));
  CK(cudaMemsetAsync(ctx->lmom.p, 0, nodes * qt->P * sizeof(double), s));
  CK(cudaMemsetAsync(ctx->pused.p, 0, nodes * sizeof(int), s));
  CK(cudaMemsetAsync(ctx->gacc.p, 0, (size_t)nh * qt->n * sizeof(double), s));
  CK(cudaMemsetAsync(ctx->counters.p, 0, sizeof(RoundCounters), s));
  u64* ns = ctx->node_state.as<u64>();
  b->inherited = ns;
  b->decided = ns + nodes;
  b->incr = ns + 2 * nodes;
  b->lbsum = ns + 3 * nodes;
  b->L = ctx->lmom.as<double>();
  b->pused = ctx->pused.as<int>();
  b->gacc = ctx->gacc.as<double>();
  b->h = ctx->hvals.as<double>();
  const float* fl = reinterpret_cast<const float*>(ctx->hvals.as<double>() + nh);
  b->inv2h2_dn = fl;
  b->inv2h2_up = fl + nh;
  b->inv_2h_up = fl + 2 * nh;
  b->c2 = fl + 3 * nh;
  b->sf = fl + 4 * nh;
  b->base_exp = &ctx->counters.as<RoundCounters>()->base_exp;
  b->status = &ctx->counters.as<RoundCounters>()->status;
  b->ku = b->kl = b->sq = b->sr = nullptr;
  b->nh = nh;
  b->eps_eff = eps_eff;
  // the expanded form of exact sums may spend a quarter of the float allowance
  b->exp_err = std::nextafter((float)(0.25 * eps_fp), 0.f);
  // lower bounds in units of the references each query can see, 2^-62
  b->loo = loo ? 1 : 0;
  b->fix_scale = std::ldexp(1.0, 62) / (double)(loo ? rt->n - 1 : rt->n);
  b->inv_fix = 1.0 / b->fix_scale;
  b->fix_scale_dn = std::nextafter((float)b->fix_scale, 0.f);
  b->inv_nr = 1.0 / (double)rt->n;
  // tau = eps_eff |R| G^l / |R_total| with G^l = lb |R_total| 2^-62
  b->tau_scale_dn = std::nextafter((float)std::ldexp(eps_eff, -62), 0.f);
  b->p_limit = std::min(qt->p_limit, rt->p_limit);
  if (ctx->sms == 0 &&
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
    return fail(ctx, DFGT_ECUDA, "dfgt_sum: device query failed");
  b->sms = ctx->sms;
  return DFGT_OK;
}

dfgt_status ensure_lists(dfgt_ctx* ctx) {
  CK(ctx->frontier[0].ensure(ctx->cap_frontier * sizeof(Pair)));
  CK(ctx->frontier[1].ensure(ctx->cap_frontier * sizeof(Pair)));
  CK(ctx->list_far.ensure(ctx->cap_lists * sizeof(Action)));
  CK(ctx->list_loc.ensure(ctx->cap_lists * sizeof(Action)));
  CK(ctx->list_f2l.ensure(ctx->cap_lists * sizeof(Action)));
  CK(ctx->list_base.ensure(ctx->cap_lists * sizeof(Pair)));
  return DFGT_OK;
}

// One kind of action list: its device buffer, its fill and the kernel that drains it.
struct ListState {
  int count = 0;
  long long total = 0;
  double ms = 0.0;       // device time of this list's kernel, all launches
  double ms_tc = 0.0;    // of which the tensor-core exact sums (D >= 6)
  bool timed = false;    // a launch is bracketed by its events, not yet read
  bool timed_tc = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr, t0 = nullptr, t1 = nullptr;
  void collect() {
    if (!timed) return;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms += t;
    timed = false;
    if (timed_tc && cudaEventElapsedTime(&t, t0, t1) == cudaSuccess) ms_tc += t;
    timed_tc = false;
  }
};

// Run the action kernel of a list over its current contents and empty it.
// Stream order makes the next round's appends start after the kernel read
// the list, so no synchronisation is needed.
dfgt_status drain(dfgt_ctx* ctx, const dfgt_tree* qt, const dfgt_tree* rt, const TravBuffers& b,
                  int which, ListState& ls, int* dcount) {
  if (ls.count == 0) return DFGT_OK;
  cudaStream_t s = ctx->stream;
  const TreeView Q = qt->view(), R = rt->view();
  if (ls.timed) {  // the previous launch of this list has finished reading by now
    CK(cudaEventSynchronize(ls.e1));
    ls.collect();
  }
  if (which != 0) {  // far field, local moments, far to local: the trees' moments and float node data
    CK(wait_ready(s, qt));
    CK(wait_ready(s, rt));
  }
  CK(cudaEventRecord(ls.e0, s));
  if (which == 0) {
    BaseScratch sc{&ctx->grp_cnt, &ctx->grp_off, &ctx->grp_r, &ctx->scan_tmp, &ctx->tc_plan};
    if (qt->d >= 6) {
      sc.tc0 = ls.t0;
      sc.tc1 = ls.t1;
      ls.timed_tc = true;
    }
    CK(launch_base(Q, R, b, ctx->list_base.as<Pair>(), ls.count, sc, s, &ctx->launches));
  }
  else if (which == 1) {
    BaseScratch sc{&ctx->grp_cnt, &ctx->grp_off, &ctx->grp_r, &ctx->scan_tmp, &ctx->tc_plan};
    CK(launch_farfield(Q, R, b, ctx->list_far.as<Action>(), ls.count, sc, s, &ctx->launches));
  } else if (which == 2) {
    BaseScratch sc{&ctx->grp_cnt, &ctx->grp_off, &ctx->grp_r, &ctx->scan_tmp, &ctx->tc_plan};
    CK(launch_local(Q, R, b, ctx->list_loc.as<Action>(), ls.count, sc, s, &ctx->launches));
  } else {
    CK(launch_f2l(Q, R, b, ctx->list_f2l.as<Action>(), ls.count, s));
    ++ctx->launches;
  }
  CK(cudaEventRecord(ls.e1, s));
  ls.timed = true;
  CK(cudaMemsetAsync(dcount, 0, sizeof(int), s));
  ls.count = 0;
  return DFGT_OK;
}

dfgt_status run_sum(dfgt_ctx* ctx, const dfgt_tree* qt, const dfgt_tree* rt, const double* h_host,
                    int nh, double eps, double* G_dev, dfgt_stats* st, bool loo = false) {
  cudaStream_t s = ctx->stream;
  const long long launches0 = ctx->launches;
  const TreeView Q = qt->view(), R = rt->view();
  const double eps_fp = float_allowance(qt, rt, eps);
  const double eps_eff = eps - eps_fp;
  const int max_rounds = qt->depth + rt->depth + 8;
  TravBuffers b;
  dfgt_status rc = setup_state(ctx, qt, rt, h_host, nh, eps_eff, eps_fp, &b, loo);
  if (rc != DFGT_OK) return rc;
  b.base_block = std::max(qt->base_block, rt->base_block);
  ctx->cap_frontier = std::max<size_t>(ctx->cap_frontier, (size_t)nh);
  rc = ensure_lists(ctx);
  if (rc != DFGT_OK) return rc;
  RoundCounters* dctr = ctx->counters.as<RoundCounters>();
  RoundCounters* hc = ctx->h_counters;
  int* dcount[4] = {&dctr->n_base, &dctr->n_far, &dctr->n_loc, &dctr->n_f2l};
  ListState lists[4];
  for (int w = 0; w < 4; ++w) {
    lists[w].e0 = ctx->ev[8 + 2 * w];
    lists[w].e1 = ctx->ev[9 + 2 * w];
  }
  lists[0].t0 = ctx->ev[16];
  lists[0].t1 = ctx->ev[17];
  int flushes = 0;
  double ms_classify = 0.0;
  CK(cudaEventRecord(ctx->ev[0], s));
  if (qt->d >= 6) {  // the bounds take the nodes' point radii, written by the moment pass
    CK(wait_ready(s, qt));
    CK(wait_ready(s, rt));
  }
  CK(launch_init_frontier(ctx->frontier[0].as<Pair>(), nh, s));
  ++ctx->launches;
  int cur = 0, nF = nh, rounds = 0;
  long long visited = 0;
  // Device-driven rounds: one cooperative launch runs rounds until the
  // frontier empties or the next round might not fit the buffers; the host
  // then drains full lists or grows the frontier and launches again.
  CK(ctx->trav_ctl.ensure(64));
  TravControl* dtc = ctx->trav_ctl.as<TravControl>();
  unsigned* dbar = reinterpret_cast<unsigned*>(ctx->trav_ctl.as<char>() + 48);
  {
    const TravControl init{nh, 0, 0, -1, 0};
    CK(cudaMemcpyAsync(dtc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  }
  TravControl htc{};
  for (int launch = 0;; ++launch) {
    if (launch > max_rounds + 8) return fail(ctx, DFGT_ETIMEOUT, "dfgt_sum: traversal did not finish");
    if ((size_t)nF > kHardCap) return fail(ctx, DFGT_ECAPACITY, "dfgt_sum: frontier exceeds 2^28 node pairs");
    // a round appends at most one item per pair to each list
    for (int w = 0; w < 4; ++w) {
      if ((size_t)lists[w].count + nF > ctx->cap_lists) {
        rc = drain(ctx, qt, rt, b, w, lists[w], dcount[w]);
        if (rc != DFGT_OK) return rc;
        ++flushes;
      }
    }
    if ((size_t)nF > ctx->cap_lists) {
      for (int w = 0; w < 4; ++w) {
        rc = drain(ctx, qt, rt, b, w, lists[w], dcount[w]);
        if (rc != DFGT_OK) return rc;
      }
      CK(cudaStreamSynchronize(s));
      ctx->cap_lists = std::max((size_t)nF, 2 * ctx->cap_lists);
      rc = ensure_lists(ctx);
      if (rc != DFGT_OK) return rc;
    }
    // both frontier buffers (and the per-pair bounds) hold at least 8 nF
    // pairs, so the frontier can grow twofold before the next return; a
    // launch that stopped because the frontier outgrew them doubles them
    const bool outgrew = 4 * (size_t)nF > ctx->cap_frontier;
    const size_t grown = outgrew ? 2 * ctx->cap_frontier : ctx->cap_frontier;
    const size_t capf = std::min<size_t>(std::max(grown, 8 * (size_t)nF), INT32_MAX);
    ctx->cap_frontier = capf;
    CK(grow_keep(ctx->frontier[cur], capf * sizeof(Pair), (size_t)nF * sizeof(Pair), s));
    CK(ctx->frontier[cur ^ 1].ensure(capf * sizeof(Pair)));
    CK(ctx->kus.ensure(4 * capf * sizeof(float)));
    b.ku = ctx->kus.as<float>();
    b.kl = b.ku + capf;
    b.sq = b.ku + 2 * capf;
    b.sr = b.ku + 3 * capf;
    CK(cudaMemsetAsync(dbar, 0, sizeof(unsigned), s));
    CK(cudaEventRecord(ctx->ev[6], s));
    CK(launch_traverse(Q, R, b, ctx->frontier[0].as<Pair>(), ctx->frontier[1].as<Pair>(), (int)capf,
                       ctx->list_far.as<Action>(), ctx->list_loc.as<Action>(), ctx->list_f2l.as<Action>(),
                       ctx->list_base.as<Pair>(), (int)ctx->cap_lists, dctr, dtc, dbar, ctx->wait, max_rounds,
                       ctx->trav_grid, s));
    ++ctx->launches;
    CK(cudaEventRecord(ctx->ev[7], s));
    CK(cudaMemcpyAsync(hc, dctr, sizeof(RoundCounters), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&htc, dtc, sizeof(htc), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    {
      float t = 0.f;
      cudaEventElapsedTime(&t, ctx->ev[6], ctx->ev[7]);
      ms_classify += t;
    }
    if (hc->status & kStTimeout) return fail(ctx, DFGT_ETIMEOUT, "dfgt_sum: a grid barrier wait timed out");
    if ((hc->status & kStOverflow) || htc.stop == kTravOverflow)
      return fail(ctx, DFGT_ECAPACITY, "dfgt_sum: work list overflow");
    if (htc.stop < 0) return fail(ctx, DFGT_ECUDA, "dfgt_sum: traversal launch did not complete");
    for (int w = 0; w < 4; ++w) lists[w].collect();
    const int got[4] = {hc->n_base, hc->n_far, hc->n_loc, hc->n_f2l};
    for (int w = 0; w < 4; ++w) {
      lists[w].total += got[w] - lists[w].count;
      lists[w].count = got[w];
    }
    nF = htc.nF;
    cur = htc.cur;
    rounds = htc.rounds;
    visited = htc.visited;
    if (htc.stop == kTravDone) break;
    if (htc.stop == kTravRounds) return fail(ctx, DFGT_ETIMEOUT, "dfgt_sum: traversal did not finish");
    // kTravRoom: drain or grow at the top of the loop and go on
    htc.stop = -1;
    CK(cudaMemcpyAsync(&dtc->stop, &htc.stop, sizeof(int), cudaMemcpyHostToDevice, s));
  }
  CK(cudaEventRecord(ctx->ev[1], s));
  for (int w = 0; w < 4; ++w) {
    rc = drain(ctx, qt, rt, b, w, lists[w], dcount[w]);
    if (rc != DFGT_OK) return rc;
  }
  // a sum that had to drain lists early leaves room for the next one
  if (flushes > 0) ctx->cap_lists = std::min(kHardCap, 2 * ctx->cap_lists);
  CK(cudaEventRecord(ctx->ev[2], s));
  rc = post(ctx, qt, b, G_dev, st);
  if (rc != DFGT_OK) return rc;
  if (hc->status & kStTimeout) return fail(ctx, DFGT_ETIMEOUT, "dfgt_sum: an exact-sum wait timed out");
  for (int w = 0; w < 4; ++w) lists[w].collect();
  if (st) {
    st->pairs_visited = visited;
    st->n_prune = (long long)hc->n_prune;
    st->n_base = lists[0].total;
    st->n_farfield = lists[1].total;
    st->n_local = lists[2].total;
    st->n_f2l = lists[3].total;
    st->base_interactions = (long long)hc->base_inter;
    st->base_expanded = (long long)hc->base_exp;
    st->farfield_terms = (long long)hc->far_terms;
    st->local_terms = (long long)hc->loc_terms;
    st->f2l_terms = (long long)hc->f2l_terms;
    st->rounds = rounds;
    st->list_flushes = flushes;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    st->ms_traverse = ms;
    st->ms_classify = ms_classify;
    cudaEventElapsedTime(&ms, ctx->ev[1], ctx->ev[2]);
    st->ms_actions = ms;
    st->ms_base = lists[0].ms;
    st->ms_base_tc = lists[0].ms_tc;
    st->ms_farfield = lists[1].ms;
    st->ms_local = lists[2].ms;
    st->ms_f2l = lists[3].ms;
    st->kernel_launches = ctx->launches - launches0;
  }
  return DFGT_OK;
}

}  // namespace

extern "C" {

dfgt_status dfgt_create(dfgt_ctx** out, int device, void* cuda_stream) {
  if (!out) return DFGT_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return DFGT_ECUDA;
  if (device < 0 || device >= ndev) return DFGT_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return DFGT_ECUDA;
  dfgt_ctx* ctx = new dfgt_ctx();
  ctx->device = device;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    ctx->own_stream = true;
  }
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_counters, sizeof(RoundCounters));
  if (e == cudaSuccess) {
    // tree arenas: a pool of our own that keeps freed memory cached
    ctx->tpool = std::make_shared<TreePool>();
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&ctx->tpool->pool, &props);
    if (e == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(ctx->tpool->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    ctx->tpool->stream = ctx->stream;
  }
  for (int i = 0; i < kCtxEvents && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->ev[i]);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->moments_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    dfgt_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? DFGT_ENOMEM : DFGT_ECUDA;
  }
  *out = ctx;
  return DFGT_OK;
}

dfgt_status dfgt_set_capacity(dfgt_ctx* ctx, int64_t frontier_pairs, int64_t list_items) {
  if (!ctx) return DFGT_EINVAL;
  if (frontier_pairs < 1 || list_items < 1 || (size_t)frontier_pairs > kHardCap ||
      (size_t)list_items > kHardCap)
    return fail(ctx, DFGT_EINVAL, "dfgt_set_capacity: need 1 <= capacity <= 2^28");
  ctx->cap_frontier = (size_t)frontier_pairs;
  ctx->cap_lists = (size_t)list_items;
  return DFGT_OK;
}

void dfgt_destroy(dfgt_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  DevBuf* bufs[] = {&ctx->scan_tmp, &ctx->counters, &ctx->hvals, &ctx->frontier[0], &ctx->frontier[1],
                    &ctx->grp_cnt, &ctx->grp_off, &ctx->grp_r, &ctx->tc_plan, &ctx->kus,
                    &ctx->list_far, &ctx->list_loc, &ctx->list_f2l, &ctx->list_base, &ctx->node_state,
                    &ctx->lmom, &ctx->pused, &ctx->gacc, &ctx->io_q, &ctx->io_r, &ctx->io_g,
                    &ctx->bf_partials, &ctx->bscratch, &ctx->bnodes, &ctx->cv_buf, &ctx->grad_buf,
                    &ctx->log_items, &ctx->log_ctr};
  for (DevBuf* b : bufs) b->release();
  if (ctx->tpool) {
    // trees that outlive the context return their arenas in default-stream order
    std::lock_guard<std::mutex> g(ctx->tpool->m);
    ctx->tpool->stream = nullptr;
  }
  ctx->tpool.reset();
  if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
  for (int i = 0; i < kCtxEvents; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->moments_done) cudaEventDestroy(ctx->moments_done);
  delete ctx;
}

long long dfgt_launch_count(const dfgt_ctx* ctx) { return ctx ? ctx->launches : -1; }

dfgt_status dfgt_test_wait_timeout(dfgt_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return DFGT_EINVAL;
  ctx->wait = BarrierCfg{};
  if (on) {
    ctx->wait.limit = 4096;  // a few milliseconds of polling
    ctx->wait.extra = 1;     // one arrival more than the grid has: no block passes
  }
  return DFGT_OK;
}

const char* dfgt_last_error(const dfgt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dfgt_status dfgt_build(dfgt_ctx* ctx, const float* points_dev, int64_t n, int d,
                       const dfgt_opts* opts, dfgt_tree** out) {
  if (!ctx || !out) return DFGT_EINVAL;
  *out = nullptr;
  if (!points_dev || n < 1 || n > (int64_t)std::numeric_limits<int>::max() / 4 || d < 1 || d > kMaxD)
    return fail(ctx, DFGT_EINVAL, "dfgt_build: need points, 1 <= n < 2^29, 1 <= d <= 32");
  if (opts && (opts->leaf_size < 0 || opts->leaf_size > kMaxLeaf || opts->p_max < 0 || opts->eps_fp < 0 ||
               opts->base_block < -1))
    return fail(ctx, DFGT_EINVAL, "dfgt_build: options out of range");
  CK(cudaSetDevice(ctx->device));
  dfgt_tree* t = new dfgt_tree();
  t->device = ctx->device;
  ctx->err.clear();
  dfgt_status rc = build_tree(ctx, points_dev, n, d, opts, t);
  if (rc != DFGT_OK) {
    delete t;
    return rc;
  }
  *out = t;
  return DFGT_OK;
}

void dfgt_tree_destroy(dfgt_tree* tree) {
  if (!tree) return;
  cudaSetDevice(tree->device);
  free_tree(tree);
  delete tree;
}

dfgt_status dfgt_sum(dfgt_ctx* ctx, const dfgt_tree* qtree, const dfgt_tree* rtree,
                     const double* h_host, int nh, double eps, double* G_dev, dfgt_stats* stats) {
  if (!ctx) return DFGT_EINVAL;
  if (!qtree || !rtree || !G_dev || qtree->d != rtree->d)
    return fail(ctx, DFGT_EINVAL, "dfgt_sum: need two trees of the same dimension and an output");
  if (bad_h(h_host, nh)) return fail(ctx, DFGT_EINVAL, "dfgt_sum: need 1..1024 finite bandwidths > 0");
  if (!(eps > 0.0 && eps < 1.0)) return fail(ctx, DFGT_EINVAL, "dfgt_sum: need 0 < eps < 1");
  if (!(float_allowance(qtree, rtree, eps) < eps))
    return fail(ctx, DFGT_EINVAL, "dfgt_sum: eps must exceed the float allowance eps_fp");
  if (qtree->device != ctx->device || rtree->device != ctx->device)
    return fail(ctx, DFGT_EINVAL, "dfgt_sum: trees live on another device");
  CK(cudaSetDevice(ctx->device));
  ctx->err.clear();
  if (stats) std::memset(stats, 0, sizeof(*stats));
  return run_sum(ctx, qtree, rtree, h_host, nh, eps, G_dev, stats);
}

dfgt_status dfgt_sum_log(dfgt_ctx* ctx, const dfgt_tree* qtree, const dfgt_tree* rtree, const double* h_host,
                         int nh, double eps, double* G_dev, double* logG_dev, dfgt_stats* stats) {
  if (!ctx) return DFGT_EINVAL;
  if (!logG_dev) return fail(ctx, DFGT_EINVAL, "dfgt_sum_log: need a log G output");
  dfgt_status rc = dfgt_sum(ctx, qtree, rtree, h_host, nh, eps, G_dev, stats);
  if (rc != DFGT_OK) return rc;
  cudaStream_t s = ctx->stream;
  CK(cudaEventRecord(ctx->ev[4], s));
  CK(wait_ready(s, rtree));
  CK(ctx->log_ctr.ensure(64));
  int* ictr = ctx->log_ctr.as<int>();
  unsigned long long* nflag = reinterpret_cast<unsigned long long*>(ctx->log_ctr.as<char>() + 8);
  int* status = ictr + 4;
  CK(cudaMemsetAsync(ctx->log_ctr.p, 0, 64, s));
  // dfgt_sum left the bandwidths in ctx->hvals
  int n_items = 0;
  CK(launch_log_pass(qtree->view(), rtree->view(), ctx->hvals.as<double>(), nh, eps, kLogFlag, G_dev, logG_dev,
                     ctx->log_items, ictr, nflag, status, s, &ctx->launches, &n_items));
  struct { unsigned long long flagged; int status; } h{};
  CK(cudaMemcpyAsync(&h.flagged, nflag, sizeof(h.flagged), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&h.status, status, sizeof(h.status), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ctx->ev[5], s));
  CK(cudaStreamSynchronize(s));
  if (h.status & kStOverflow) return fail(ctx, DFGT_ECAPACITY, "dfgt_sum_log: reference tree too deep for the walk");
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]);
    stats->ms_log = ms;
    stats->log_queries = (long long)h.flagged;
    stats->kernel_launches += 3;
  }
  return DFGT_OK;
}

dfgt_status dfgt_sum_loo(dfgt_ctx* ctx, const dfgt_tree* tree, const double* h_host, int nh, double eps,
                         double* S_dev, dfgt_stats* stats) {
  if (!ctx) return DFGT_EINVAL;
  if (!tree || !S_dev || tree->n < 2)
    return fail(ctx, DFGT_EINVAL, "dfgt_sum_loo: need a tree of at least 2 points and an output");
  if (bad_h(h_host, nh)) return fail(ctx, DFGT_EINVAL, "dfgt_sum_loo: need 1..1024 finite bandwidths > 0");
  if (!(eps > 0.0 && eps < 1.0)) return fail(ctx, DFGT_EINVAL, "dfgt_sum_loo: need 0 < eps < 1");
  if (!(float_allowance(tree, tree, eps) < eps)) return fail(ctx, DFGT_EINVAL, "dfgt_sum_loo: eps must exceed the float allowance eps_fp");
  if (tree->device != ctx->device) return fail(ctx, DFGT_EINVAL, "dfgt_sum_loo: the tree lives on another device");
  CK(cudaSetDevice(ctx->device));
  ctx->err.clear();
  if (stats) std::memset(stats, 0, sizeof(*stats));
  return run_sum(ctx, tree, tree, h_host, nh, eps, S_dev, stats, true);
}

dfgt_status dfgt_cv_scores(dfgt_ctx* ctx, const dfgt_tree* tree, const double* h_host, int nh, double eps,
                           double* cv_lk, double* cv_ls, double* lk_bound, double* ls_bound,
                           dfgt_stats* stats) {
  if (!ctx) return DFGT_EINVAL;
  if (!tree || !cv_lk || !cv_ls || tree->n < 2)
    return fail(ctx, DFGT_EINVAL, "dfgt_cv_scores: need a tree of at least 2 points and score outputs");
  if (bad_h(h_host, nh) || nh > 512)
    return fail(ctx, DFGT_EINVAL, "dfgt_cv_scores: need 1..512 finite bandwidths > 0");
  const int n = (int)tree->n, d = tree->d;
  std::vector<double> h2(2 * (size_t)nh), norm(2 * (size_t)nh);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < nh; ++k) {
    h2[k] = h_host[k];
    h2[nh + k] = std::sqrt(2.0) * h_host[k];
  }
  for (int k = 0; k < 2 * nh; ++k) norm[k] = (double)(n - 1) * std::pow(2.0 * pi * h2[k] * h2[k], 0.5 * d);
  CK(cudaSetDevice(ctx->device));
  CK(ctx->io_g.ensure(2 * (size_t)nh * n * sizeof(double)));
  dfgt_status rc = dfgt_sum_loo(ctx, tree, h2.data(), 2 * nh, eps, ctx->io_g.as<double>(), stats);
  if (rc != DFGT_OK) return rc;
  const int nblk = std::max(1, std::min(304, (n + 1023) / 1024));
  const size_t nnorm = 2 * (size_t)nh, npart = (size_t)nh * nblk * 4, nout = (size_t)nh * 4;
  CK(ctx->cv_buf.ensure((nnorm + npart + nout) * sizeof(double)));
  double* dnorm = ctx->cv_buf.as<double>();
  double* dpart = dnorm + nnorm;
  double* dout = dpart + npart;
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(dnorm, norm.data(), nnorm * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(launch_cv_scores(ctx->io_g.as<double>(), n, nh, dnorm, eps, dpart, nblk, dout, s, &ctx->launches));
  std::vector<double> out(nout);
  CK(cudaMemcpyAsync(out.data(), dout, nout * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < nh; ++k) {
    cv_lk[k] = out[4 * k];
    cv_ls[k] = out[4 * k + 2];
    if (lk_bound) lk_bound[k] = out[4 * k + 1];
    if (ls_bound) ls_bound[k] = out[4 * k + 3];
  }
  return DFGT_OK;
}

dfgt_status dfgt_cv_grad(dfgt_ctx* ctx, const float* x_dev, int64_t n64, int d, const double* h_host, int nh,
                         double* cv, double* dcv_dlogh, double* dcv_dx_dev) {
  if (!ctx) return DFGT_EINVAL;
  if (!x_dev || !cv || !dcv_dlogh || n64 < 2 || n64 > (int64_t)std::numeric_limits<int>::max() / 4 || d < 1 ||
      d > kMaxD)
    return fail(ctx, DFGT_EINVAL, "dfgt_cv_grad: need points, 2 <= n < 2^29, 1 <= d <= 32 and score outputs");
  if (bad_h(h_host, nh) || nh > 512)
    return fail(ctx, DFGT_EINVAL, "dfgt_cv_grad: need 1..512 finite bandwidths > 0");
  const int n = (int)n64;
  const int nb = (n + 255) / 256;
  const size_t nS = (size_t)n, nP = (size_t)n * d;
  CK(cudaSetDevice(ctx->device));
  CK(ctx->grad_buf.ensure((2 * nS + 2 * nP + 2 * (size_t)nb + 2 * (size_t)nh) * sizeof(double)));
  double* S = ctx->grad_buf.as<double>();
  double* A = S + nS;
  double* P = A + nS;
  double* Y = P + nP;
  double* part = Y + nP;
  double* out = part + 2 * (size_t)nb;
  cudaStream_t s = ctx->stream;
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < nh; ++k) {
    double* dx = dcv_dx_dev ? dcv_dx_dev + (size_t)k * nP : nullptr;
    CK(launch_cv_grad(x_dev, n, d, h_host[k], S, P, A, Y, part, out + 2 * k, dx, s, &ctx->launches));
  }
  std::vector<double> o(2 * (size_t)nh);
  CK(cudaMemcpyAsync(o.data(), out, o.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < nh; ++k) {
    const double h = h_host[k];
    const double lognorm = std::log((double)(n - 1)) + 0.5 * d * std::log(2.0 * pi * h * h);
    cv[k] = o[2 * k] / n - lognorm;
    dcv_dlogh[k] = o[2 * k + 1] / n - d;
  }
  return DFGT_OK;
}

dfgt_status dfgt_autotune(dfgt_ctx* ctx, const float* points_dev, int64_t n, int d, const double* h_host,
                          int nh, double eps, int trials, dfgt_opts* best, double* best_ms) {
  if (!ctx) return DFGT_EINVAL;
  if (!points_dev || !best || n < 1 || n > (int64_t)std::numeric_limits<int>::max() / 4 || d < 1 || d > kMaxD ||
      trials < 1 || trials > 16)
    return fail(ctx, DFGT_EINVAL, "dfgt_autotune: need points, 1 <= n < 2^29, 1 <= d <= 32, 1 <= trials <= 16");
  if (bad_h(h_host, nh)) return fail(ctx, DFGT_EINVAL, "dfgt_autotune: need 1..1024 finite bandwidths > 0");
  if (!(eps > 0.0 && eps < 1.0)) return fail(ctx, DFGT_EINVAL, "dfgt_autotune: need 0 < eps < 1");
  CK(cudaSetDevice(ctx->device));
  CK(ctx->io_g.ensure((size_t)nh * n * sizeof(double)));
  // candidates: leaf sizes, exact-sum thresholds (the block |Q| |R| of one
  // exact sum) and, unless the caller fixed it, the expansion order limit
  // p_max and one below it (fewer coefficients per node against fewer
  // pairs that a series can take)
  const int leaves[] = {32, 64, 96, 128, 160, 192};
  const long long blocks[] = {2048, 4096, 8192};
  dfgt_opts start = *best;
  const int pm_table = pmax_of(d);
  int orders[2] = {start.p_max > 0 ? std::min(start.p_max, pm_table) : pm_table, 0};
  int norders = 1;
  if (start.p_max <= 0 && pm_table > 1) orders[norders++] = pm_table - 1;
  double best_t = 1e300;
  dfgt_opts chosen = start;
  for (int oi = 0; oi < norders; ++oi)
  for (int leaf : leaves) {
    if (leaf > kMaxLeaf) continue;
    for (long long bb : blocks) {
      dfgt_opts o = start;
      o.leaf_size = leaf;
      o.base_block = bb;
      o.p_max = orders[oi];
      double tmin = 1e300;
      for (int rep = 0; rep <= trials; ++rep) {  // the first run warms up and is not counted
        CK(cudaEventRecord(ctx->ev[4], ctx->stream));
        dfgt_tree* t = nullptr;
        dfgt_status rc = dfgt_build(ctx, points_dev, n, d, &o, &t);
        if (rc != DFGT_OK) return rc;
        rc = dfgt_sum(ctx, t, t, h_host, nh, eps, ctx->io_g.as<double>(), nullptr);
        dfgt_tree_destroy(t);
        if (rc != DFGT_OK) return rc;
        CK(cudaEventRecord(ctx->ev[5], ctx->stream));
        CK(cudaEventSynchronize(ctx->ev[5]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]));
        if (rep > 0) tmin = std::min(tmin, (double)ms);
      }
      if (tmin < best_t) {
        best_t = tmin;
        chosen = o;
      }
    }
  }
  *best = chosen;
  if (best_ms) *best_ms = best_t;
  return DFGT_OK;
}

dfgt_status dfgt_sum_bruteforce(dfgt_ctx* ctx, const float* q_dev, int64_t nq, const float* r_dev,
                                int64_t nr, int d, const double* h_host, int nh, double* G_dev) {
  if (!ctx) return DFGT_EINVAL;
  if (!q_dev || !r_dev || !G_dev || nq < 1 || nr < 1 || nq > std::numeric_limits<int>::max() ||
      nr > std::numeric_limits<int>::max() || d < 1 || d > kMaxD)
    return fail(ctx, DFGT_EINVAL, "dfgt_sum_bruteforce: bad sizes or pointers");
  if (bad_h(h_host, nh)) return fail(ctx, DFGT_EINVAL, "dfgt_sum_bruteforce: need 1..1024 finite bandwidths > 0");
  CK(cudaSetDevice(ctx->device));
  ctx->err.clear();
  CK(launch_bruteforce(q_dev, (int)nq, r_dev, (int)nr, d, h_host, nh, G_dev, ctx->bf_partials,
                       ctx->stream, &ctx->launches));
  CK(cudaStreamSynchronize(ctx->stream));
  return DFGT_OK;
}

dfgt_status dfgt_kde_host(dfgt_ctx* ctx, const float* q_host, int64_t nq, const float* r_host,
                          int64_t nr, int d, const double* h_host, int nh, double eps,
                          const dfgt_opts* opts, double* G_host, dfgt_stats* stats) {
  if (!ctx) return DFGT_EINVAL;
  if (!q_host || !r_host || !G_host || nq < 1 || nr < 1 || d < 1 || d > kMaxD)
    return fail(ctx, DFGT_EINVAL, "dfgt_kde_host: bad sizes or pointers");
  if (bad_h(h_host, nh)) return fail(ctx, DFGT_EINVAL, "dfgt_kde_host: need 1..1024 finite bandwidths > 0");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const bool same = (q_host == r_host) && (nq == nr);
  CK(ctx->io_q.ensure((size_t)nq * d * sizeof(float)));
  CK(cudaMemcpyAsync(ctx->io_q.p, q_host, (size_t)nq * d * sizeof(float), cudaMemcpyHostToDevice, s));
  if (!same) {
    CK(ctx->io_r.ensure((size_t)nr * d * sizeof(float)));
    CK(cudaMemcpyAsync(ctx->io_r.p, r_host, (size_t)nr * d * sizeof(float), cudaMemcpyHostToDevice, s));
  }
  CK(ctx->io_g.ensure((size_t)nh * nq * sizeof(double)));
  dfgt_tree *qt = nullptr, *rt = nullptr;
  dfgt_status rc = dfgt_build(ctx, ctx->io_q.as<float>(), nq, d, opts, &qt);
  if (rc == DFGT_OK) {
    if (same) rt = qt;
    else rc = dfgt_build(ctx, ctx->io_r.as<float>(), nr, d, opts, &rt);
  }
  if (rc == DFGT_OK) rc = dfgt_sum(ctx, qt, rt, h_host, nh, eps, ctx->io_g.as<double>(), stats);
  if (rc == DFGT_OK) {
    cudaError_t e = cudaMemcpyAsync(G_host, ctx->io_g.p, (size_t)nh * nq * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = fail(ctx, DFGT_ECUDA, std::string("dfgt_kde_host copy-out: ") + cudaGetErrorString(e));
  }
  if (rt && rt != qt) dfgt_tree_destroy(rt);
  if (qt) dfgt_tree_destroy(qt);
  return rc;
}

dfgt_status dfgt_tree_get_info(const dfgt_tree* t, dfgt_tree_info* out) {
  if (!t || !out) return DFGT_EINVAL;
  out->n_points = t->n;
  out->d = t->d;
  out->n_nodes = t->nn;
  out->n_leaves = t->nleaves;
  out->depth = t->depth;
  out->leaf_size = t->leaf;
  out->p_max = t->pm;
  out->n_coeff = t->P;
  out->ms_levels = out->ms_moments = -1.0;
  if (cudaSetDevice(t->device) != cudaSuccess) return DFGT_ECUDA;
  if (t->ready && cudaEventSynchronize(t->ready) != cudaSuccess) return DFGT_ECUDA;
  float ms = 0.f;
  if (t->tev[0] && t->tev[1] && cudaEventElapsedTime(&ms, t->tev[0], t->tev[1]) == cudaSuccess) out->ms_levels = ms;
  if (t->tev[2] && t->tev[3] && cudaEventElapsedTime(&ms, t->tev[2], t->tev[3]) == cudaSuccess) out->ms_moments = ms;
  return DFGT_OK;
}

dfgt_status dfgt_tree_export(const dfgt_tree* t, int32_t* perm, float* lo, float* hi,
                             int32_t* begin, int32_t* count, int32_t* left, double* moments, float* radius) {
  if (!t) return DFGT_EINVAL;
  if (cudaSetDevice(t->device) != cudaSuccess) return DFGT_ECUDA;
  if (t->ready && cudaEventSynchronize(t->ready) != cudaSuccess) return DFGT_ECUDA;
  struct Item { void* dst; const void* src; size_t bytes; } items[] = {
      {perm, t->perm, (size_t)t->n * sizeof(int)},
      {lo, t->lo, (size_t)t->nn * t->d * sizeof(float)},
      {hi, t->hi, (size_t)t->nn * t->d * sizeof(float)},
      {begin, t->beg, (size_t)t->nn * sizeof(int)},
      {count, t->cnt, (size_t)t->nn * sizeof(int)},
      {left, t->left, (size_t)t->nn * sizeof(int)},
      {moments, t->mom, (size_t)t->nn * t->P * sizeof(double)},
      {radius, t->rad, (size_t)t->nn * sizeof(float)},
  };
  for (const Item& it : items)
    if (it.dst && cudaMemcpy(it.dst, it.src, it.bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
      return DFGT_ECUDA;
  return DFGT_OK;
}

dfgt_status dfgt_apply_pairs(dfgt_ctx* ctx, const dfgt_tree* qt, const dfgt_tree* rt,
                             const int32_t* qnode, const int32_t* rnode, const int32_t* action,
                             const int32_t* order, int n, double h, double* G_dev, dfgt_stats* stats) {
  if (!ctx) return DFGT_EINVAL;
  if (!qt || !rt || !G_dev || qt->d != rt->d || n < 0 || (n > 0 && (!qnode || !rnode || !action)))
    return fail(ctx, DFGT_EINVAL, "dfgt_apply_pairs: bad arguments");
  if (bad_h(&h, 1)) return fail(ctx, DFGT_EINVAL, "dfgt_apply_pairs: need a finite bandwidth > 0");
  std::vector<Pair> prune, base;
  std::vector<Action> far, loc, f2l;
  for (int i = 0; i < n; ++i) {
    const int q = qnode[i], r = rnode[i], a = action[i];
    const int p = order ? order[i] : 1;
    if (q < 0 || q >= qt->nn || r < 0 || r >= rt->nn)
      return fail(ctx, DFGT_EINVAL, "dfgt_apply_pairs: node index out of range");
    if (a == DFGT_ACT_PRUNE) prune.push_back(Pair{q, r, 0, 0});
    else if (a == DFGT_ACT_BASE) base.push_back(Pair{q, r, 0, 0});
    else if (a >= DFGT_ACT_FARFIELD && a <= DFGT_ACT_F2L) {
      if (p < 1 || p > qt->pm) return fail(ctx, DFGT_EINVAL, "dfgt_apply_pairs: order out of range");
      (a == DFGT_ACT_FARFIELD ? far : a == DFGT_ACT_LOCAL ? loc : f2l).push_back(Action{q, r, 0, p});
    } else {
      return fail(ctx, DFGT_EINVAL, "dfgt_apply_pairs: unknown action");
    }
  }
  CK(cudaSetDevice(ctx->device));
  ctx->err.clear();
  cudaStream_t s = ctx->stream;
  TravBuffers b;
  CK(wait_ready(s, qt));
  CK(wait_ready(s, rt));
  // exact sums here take the trees' float allowance, or the smallest automatic one
  dfgt_status rc = setup_state(ctx, qt, rt, &h, 1, 0.5, float_allowance(qt, rt, 0.0), &b);
  if (rc != DFGT_OK) return rc;
  const size_t need = std::max<size_t>({prune.size(), base.size(), far.size(), loc.size(), f2l.size(), 1});
  ctx->cap_lists = std::max(ctx->cap_lists, need);
  ctx->cap_frontier = std::max(ctx->cap_frontier, need);
  rc = ensure_lists(ctx);
  if (rc != DFGT_OK) return rc;
  auto up = [&](DevBuf& dst, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst.p, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  CK(up(ctx->frontier[0], prune.data(), prune.size() * sizeof(Pair)));
  CK(up(ctx->list_base, base.data(), base.size() * sizeof(Pair)));
  CK(up(ctx->list_far, far.data(), far.size() * sizeof(Action)));
  CK(up(ctx->list_loc, loc.data(), loc.size() * sizeof(Action)));
  CK(up(ctx->list_f2l, f2l.data(), f2l.size() * sizeof(Action)));
  const TreeView Q = qt->view(), R = rt->view();
  CK(launch_prune_apply(Q, R, b, ctx->frontier[0].as<Pair>(), (int)prune.size(), s));
  BaseScratch sc{&ctx->grp_cnt, &ctx->grp_off, &ctx->grp_r, &ctx->scan_tmp, &ctx->tc_plan};
  CK(launch_base(Q, R, b, ctx->list_base.as<Pair>(), (int)base.size(), sc, s, &ctx->launches));
  CK(launch_farfield(Q, R, b, ctx->list_far.as<Action>(), (int)far.size(), sc, s, &ctx->launches));
  CK(launch_local(Q, R, b, ctx->list_loc.as<Action>(), (int)loc.size(), sc, s, &ctx->launches));
  CK(launch_f2l(Q, R, b, ctx->list_f2l.as<Action>(), (int)f2l.size(), s));
  CK(cudaEventRecord(ctx->ev[2], s));
  rc = post(ctx, qt, b, G_dev, nullptr);
  if (rc != DFGT_OK) return rc;
  if (ctx->h_counters->status & kStTimeout) return fail(ctx, DFGT_ETIMEOUT, "dfgt_apply_pairs: an exact-sum wait timed out");
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    long long inter = 0;
    std::vector<int> qc(qt->nn), rc2(rt->nn);
    CK(cudaMemcpy(qc.data(), qt->cnt, qc.size() * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rc2.data(), rt->cnt, rc2.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (const Pair& p : base) inter += (long long)qc[p.q] * rc2[p.r];
    stats->n_base = (long long)base.size();
    stats->base_interactions = inter;
    stats->base_expanded = (long long)ctx->h_counters->base_exp;
  }
  return DFGT_OK;
}

dfgt_status dfgt_grad(dfgt_ctx* ctx, const float* x_dev, int64_t n, int d, const double* h_host, int nh,
                      double* cv, double* dcv_dlogh, double* dcv_dx_dev) {
  return dfgt_cv_grad(ctx, x_dev, n, d, h_host, nh, cv, dcv_dlogh, dcv_dx_dev);
}

}  // extern "C"
