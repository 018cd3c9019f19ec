// base_tc.cu -- exact sums (DFGTBase, Section 3.6) for D >= 6 on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory).  The form, its error bound and the choice of runs:
// base_hd_forms.cuh.
//
// k_tc_plan takes each run of the sorted base list (one bandwidth, one
// query node: one key of the counting sort), decides whether it takes the
// tensor form, marks its entries (k_base_hd skips them) and lists it as
// work items of up to kItemEntries entries with its scales.
//
// k_base_tc is persistent: each CTA takes a contiguous range of work items
// of about equal cost (the plan's one packed atomic per run gives every item
// its index and the summed cost before it).  Four producer warps stage the
// operands in shared memory; the producer that stages a tile's last row
// (counted by an acquire-release shared counter) issues its MMAs, so no
// producer waits for another.  Four consumer warps read the results back
// from tensor memory and sum the exponentials.  Per item and block of up to 128
// queries, producer thread p stages query row p of A: the float16 splits
// of W_q 2^a = Wh + Wl (W_q = -2c q~) laid out as Wh | Wh | Wl | 2^s 2^s
// along K; per tile of 128 references it stages reference row p of B:
// rh | rl | rh | Bh Bl (r~ 2^b = rh + rl, B_r 2^(a+b-s) = Bh + Bl).  So one
// D = A B^T of K = 3 DM + 2 (padded to whole K16 steps) gives, per (query,
// reference), 2^(a+b) (W_q . r~ + B_r) = 2^(a+b) (x - A_q).  Both operands
// are K-major without swizzle (8 x 16-byte core matrices: 128 bytes between
// 8-row groups, 2048 bytes between K groups of 8); D is float32 in tensor
// memory, lane = query row, column = reference.  Two accumulators and two
// B buffers alternate: the MMA of tile g + 1 runs while the consumers read
// tile g (tcgen05.ld, 64 columns at a time) and add 2^(D 2^-(a+b) + A_q)
// with ex2.approx into Kahan-compensated row sums.  mbarriers order the
// roles: mma_done[b] (tcgen05.commit) tells the consumers a tile is in
// accumulator b, acc_free[b] (128 consumer arrivals) tells the producers
// that accumulator b and B buffer b may be reused.  Every wait is bounded
// and reports kStTimeout.
#include <cuda_fp16.h>

#include <algorithm>

#include "base_hd_forms.cuh"
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kTcThreads = 256;   // warps 0-3 consumers (tensor-memory lanes 0..127 = query rows), 4-7 producers
constexpr int kTcCons = 128;      // consumer threads
constexpr int kTcRows = 128;      // queries per block (MMA M) and references per tile (MMA N)
constexpr int kTcCols = 2 * kTcRows;  // tensor-memory columns: two accumulators
constexpr long long kTcWaitLimit = 1LL << 20;  // mbarrier polls before giving up
constexpr int kTcSmemFloor = 78 * 1024;  // dynamic shared memory per CTA: at most two CTAs per SM,
                                         // so their 2 x 256 columns of tensor memory always fit
constexpr int kTcCtasPerSm = 2;

template <int DM>
struct TcShape {
  static constexpr int K = ((3 * DM + 2) + 15) / 16 * 16;  // K slots, whole K16 steps
  static constexpr int KC = K / 16;                         // chained MMA steps
  static constexpr int TILE = kTcRows * K * 2;              // bytes of one operand tile
  static constexpr int SMEM = 3 * TILE;                     // A and two B tiles
  static_assert(tc_chunks(DM) == KC, "the chained steps of the error bound");
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = bytes between
// K-adjacent core matrices, sbo = bytes between 8-row groups.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: float32 D, float16 A and B, both
// K-major, N = M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(kTcRows >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ unsigned h2u(__half2 h) {
  unsigned u;
  memcpy(&u, &h, sizeof u);
  return u;
}

// (v.x, v.y) = hi + lo + err per element, |err| <= 2^-22 |v| while lo is normal
__device__ __forceinline__ void split2(float a, float b, unsigned& hi, unsigned& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 f = __half22float2(h);
  hi = h2u(h);
  lo = h2u(__floats2half2_rn(a - f.x, b - f.y));
}

__device__ __forceinline__ float pow2i(int e) { return __int_as_float((127 + e) << 23); }

// Byte offset of K group kg (8 slots) of row `row` in a 128-row tile.
__device__ __forceinline__ uint32_t tc_off(int row, int kg) {
  return (uint32_t)((kg * (kTcRows / 8) + (row >> 3)) * 128 + (row & 7) * 16);
}

// Write one row of an operand tile: parts p0 | p1 | p2 (DM float16 each, as
// DM/2 words) and the two norm slots (t0, t1), zeros after.
template <int DM>
__device__ __forceinline__ void put_row(unsigned char* tile, int row, const unsigned* p0, const unsigned* p1,
                                        const unsigned* p2, unsigned norm) {
  constexpr int G = DM / 8;  // K groups per part
#pragma unroll
  for (int g = 0; g < G; ++g) {
    *reinterpret_cast<uint4*>(tile + tc_off(row, g)) = make_uint4(p0[4 * g], p0[4 * g + 1], p0[4 * g + 2], p0[4 * g + 3]);
    *reinterpret_cast<uint4*>(tile + tc_off(row, G + g)) =
        make_uint4(p1[4 * g], p1[4 * g + 1], p1[4 * g + 2], p1[4 * g + 3]);
    *reinterpret_cast<uint4*>(tile + tc_off(row, 2 * G + g)) =
        make_uint4(p2[4 * g], p2[4 * g + 1], p2[4 * g + 2], p2[4 * g + 3]);
  }
  *reinterpret_cast<uint4*>(tile + tc_off(row, 3 * G)) = make_uint4(norm, 0u, 0u, 0u);
#pragma unroll
  for (int g = 3 * G + 1; g < TcShape<DM>::K / 8; ++g) *reinterpret_cast<uint4*>(tile + tc_off(row, g)) = make_uint4(0u, 0u, 0u, 0u);
}

template <int DM>
__device__ __forceinline__ void zero_row(unsigned char* tile, int row) {
#pragma unroll
  for (int g = 0; g < TcShape<DM>::K / 8; ++g) *reinterpret_cast<uint4*>(tile + tc_off(row, g)) = make_uint4(0u, 0u, 0u, 0u);
}

// DM coordinates of a tree row minus the centre m
template <int DM>
__device__ __forceinline__ void centred(const float* __restrict__ p, int dp, const float* m, float* v) {
#pragma unroll
  for (int k4 = 0; k4 < DM / 4; ++k4) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (4 * k4 < dp) a = __ldg(reinterpret_cast<const float4*>(p) + k4);
    v[4 * k4] = a.x - m[4 * k4];
    v[4 * k4 + 1] = a.y - m[4 * k4 + 1];
    v[4 * k4 + 2] = a.z - m[4 * k4 + 2];
    v[4 * k4 + 3] = a.w - m[4 * k4 + 3];
  }
}

// Wait for the phase of parity `phase` of an mbarrier to complete: at most
// kTcWaitLimit polls, each suspending the thread for at most 1 us, so about
// a second in all before it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase), "r"(1000u)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void kahan(float& S, float& C, float v) {
  const float y = v - C;
  const float t = S + y;
  C = (t - S) - y;
  S = t;
}

// Sum of squares by pairwise (tree) addition: relative error at most
// (log2(DM) + 1) u, with DM - 1 adds.
template <int DM>
__device__ __forceinline__ float sumsq(const float* v) {
  float t[DM];
#pragma unroll
  for (int k = 0; k < DM; ++k) t[k] = v[k] * v[k];
#pragma unroll
  for (int w = DM / 2; w >= 1; w >>= 1)
#pragma unroll
    for (int k = 0; k < w; ++k) t[k] += t[k + w];
  return t[0];
}

// tcgen05.ld of 32 columns into r (asynchronous until tc_wait32)
__device__ __forceinline__ void tc_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Wait for this thread's outstanding tcgen05.ld; r is threaded through so
// that no use of it is scheduled before the wait.
__device__ __forceinline__ void tc_wait32(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// Sum of 2^(S sout + Aq) over the first `lim` of 32 columns (packed f32x2
// FMA and adds, four independent partial sums).
__device__ __forceinline__ float ex2_sum32(const uint32_t (&r)[32], float sout, float Aq, int lim) {
  const float2 so2 = make_float2(sout, sout), aq2 = make_float2(Aq, Aq);
  float2 p2[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) p2[u] = make_float2(0.f, 0.f);
  if (lim >= 32) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float2 x = __ffma2_rn(make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])), so2, aq2);
      p2[j & 3] = __fadd2_rn(p2[j & 3], make_float2(ex2_approx(x.x), ex2_approx(x.y)));
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float2 x = __ffma2_rn(make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1])), so2, aq2);
      const float e0 = 2 * j < lim ? ex2_approx(x.x) : 0.f, e1 = 2 * j + 1 < lim ? ex2_approx(x.y) : 0.f;
      p2[j & 3] = __fadd2_rn(p2[j & 3], make_float2(e0, e1));
    }
  }
  const float2 t = __fadd2_rn(__fadd2_rn(p2[0], p2[1]), __fadd2_rn(p2[2], p2[3]));
  return t.x + t.y;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Shared-memory counter increment with acquire-release order at block scope:
// each producer's staged row (made visible to the async proxy before) is
// ordered before the MMAs of whichever producer sees the count complete.
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* c) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;" : "=r"(old) : "r"(smem_addr(c)) : "memory");
  return old;
}

// barrier of the four producer warps only
__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// barrier of the four producer warps only, returning the AND of v over them
__device__ __forceinline__ bool producers_sync_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.b32 p, %1, 0;\nbar.red.and.pred q, 1, 128, p;\nselp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

constexpr int kItemEntries = 256;  // base entries per work item at most

// One work item: up to kItemEntries consecutive entries of one tensor-form run.
struct TcItem {
  int i0, ne;        // entries [i0, i0 + ne) of the sorted list
  int hidx, qnode;   // bandwidth, query node
  int qb, qn, tot;   // first query, queries, references of the item
  int a, b, s;       // scales (the run's)
  int pad;
  unsigned long long cpre;  // summed cost of the items before this one
};

// Work of an item in tile units: each 128-query block streams the item's
// reference tiles, plus about one tile of setup.
__device__ __forceinline__ unsigned long long item_cost(int qn, int tot) {
  return (unsigned long long)((qn + kTcRows - 1) / kTcRows) * (unsigned long long)((tot + kTcRows - 1) / kTcRows + 1);
}

// The plan's counter packs the item count (low kItemCountBits; lists hold at
// most 2^28 entries) and the summed cost of the items (the rest, 2^35 tile
// units), so that one atomic gives an item both its index and its cost prefix,
// in the same order. A sum that would pass 2^35 sets the plan's overflow word
// and the CTAs then take the items in turn instead.
constexpr int kItemCountBits = 29;
constexpr unsigned long long kItemCountMask = (1ull << kItemCountBits) - 1;

// Plan: one warp per key (bandwidth, query node) of the counting sort; the
// key's entries are [end - cnt, end).
template <int DM>
__global__ void __launch_bounds__(256) k_tc_plan(TreeView Q, TreeView R, const int* __restrict__ rsorted,
                                                 const int* __restrict__ cnt, const int* __restrict__ end, int nkeys,
                                                 const float* __restrict__ c2v, const float* __restrict__ inv2h2_up,
                                                 float exp_err, unsigned char* __restrict__ tcflag,
                                                 TcItem* __restrict__ items, unsigned long long* __restrict__ plan_ctr,
                                                 unsigned long long* __restrict__ tc_ctr) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long key = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (key >= nkeys) return;
  const int c = cnt[key];
  if (c == 0) return;
  const int b0 = end[key] - c;
  const int hidx = (int)(key / Q.nn), q = (int)(key - (long)hidx * Q.nn);
  float mc[DM];
  const float rho2 = hd_query_bounds<DM>(Q, q, mc);  // once per run
  float f2 = 0.f;
  bool self = false;
  long long tot = 0;
  for (int i = lane; i < c; i += 32) {
    const int rv = rsorted[b0 + i];
    const int r = rv & kNodeMask;
    self |= ((rv >> kNodeBits) & kSelfFlag) != 0;
    f2 = fmaxf(f2, hd_entry_far2<DM>(R, r, mc));
    tot += R.cnt[r];
  }
  f2 = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(f2)));
  self = __any_sync(FULL, self);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
  const int qn = Q.cnt[q];
  HtScale sc;
  const bool tc = hd_tensor_form(Q.d, tc_chunks(DM), rho2, f2, inv2h2_up[hidx], c2v[hidx], self, qn, exp_err, &sc);
  for (int i = lane; i < c; i += 32) tcflag[b0 + i] = tc ? 1 : 0;
  if (!tc) return;
  const int nparts = (c + kItemEntries - 1) / kItemEntries;
  // the parts' references: counted once for the summed cost, again for the items
  auto part_refs = [&](int j) {
    const int i0 = b0 + j * kItemEntries, ne = min(kItemEntries, c - j * kItemEntries);
    int pt = 0;
    for (int i = lane; i < ne; i += 32) pt += R.cnt[rsorted[i0 + i] & kNodeMask];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pt += __shfl_xor_sync(FULL, pt, o);
    return pt;
  };
  unsigned long long cost = 0;
  for (int j = 0; j < nparts; ++j) cost += item_cost(qn, part_refs(j));
  unsigned long long old = 0;
  if (lane == 0) {
    old = atomicAdd(plan_ctr, (cost << kItemCountBits) | (unsigned long long)nparts);
    if ((old >> kItemCountBits) + cost >= (1ull << (64 - kItemCountBits)) || cost >= (1ull << (64 - kItemCountBits)))
      atomicOr(reinterpret_cast<unsigned int*>(plan_ctr + 1), 1u);
    atomicAdd(tc_ctr, (unsigned long long)qn * (unsigned long long)tot);
  }
  old = __shfl_sync(FULL, old, 0);
  const int k = (int)(old & kItemCountMask);
  unsigned long long cpre = old >> kItemCountBits;
  const int qb = Q.beg[q];
  for (int j = 0; j < nparts; ++j) {
    const int i0 = b0 + j * kItemEntries, ne = min(kItemEntries, c - j * kItemEntries);
    const int pt = part_refs(j);
    if (lane == 0) items[k + j] = TcItem{i0, ne, hidx, q, qb, qn, pt, sc.a, sc.b, sc.s, 0, cpre};
    cpre += item_cost(qn, pt);
  }
}

// Items [first, last) of CTA c of G: those whose cost interval has its middle
// in [c T / G, (c + 1) T / G), T the summed cost (items are in prefix order,
// so each CTA takes a contiguous range of about T / G).
__device__ __forceinline__ int items_owner(const TcItem& it, unsigned long long T, int G) {
  const unsigned long long mid2 = 2 * it.cpre + item_cost(it.qn, it.tot);
  return (int)(mid2 * (unsigned long long)G / (2 * T));
}
__device__ int items_lower_bound(const TcItem* items, int n, unsigned long long T, int G, int c) {
  int lo = 0, hi = n;  // first item whose owner is >= c
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (items_owner(items[mid], T, G) < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int DM>
__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm)
    k_base_tc(TreeView Q, TreeView R, const int* __restrict__ rsorted, const TcItem* __restrict__ items,
              const unsigned long long* __restrict__ plan_ctr, const float* __restrict__ c2v, double* __restrict__ gacc,
              int* __restrict__ status) {
  using SH = TcShape<DM>;
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* const tA = dsm;
  unsigned char* const tB0 = dsm + SH::TILE;
  __shared__ int sOff[kItemEntries], sRb[kItemEntries];
  __shared__ int sAbort;   // a wait ran out: every role leaves at its next check
  __shared__ uint32_t sTmem;
  __shared__ __align__(8) uint64_t sDone[2], sFree[2];  // mma_done, acc_free
  __shared__ uint32_t sArr[2];  // producer rows staged into B buffer 0 / 1 (all tiles so far)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned FULL = 0xffffffffu;
  const unsigned long long ctr = *plan_ctr;
  const int n_items = (int)(ctr & kItemCountMask);
  const unsigned long long T = ctr >> kItemCountBits;
  const bool in_turn = *reinterpret_cast<const unsigned int*>(plan_ctr + 1) != 0;
  if (n_items == 0) return;
  __shared__ int sRange[2];
  if (tid < 2)
    sRange[tid] = in_turn ? 0 : items_lower_bound(items, n_items, T, gridDim.x, blockIdx.x + tid);
  __syncthreads();
  // a contiguous range of about T / G, or (after an overflow) every G-th item
  const int it0 = in_turn ? (int)blockIdx.x : sRange[0], it1 = in_turn ? n_items : sRange[1];
  const int istep = in_turn ? (int)gridDim.x : 1;
  if (it0 >= it1) return;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sTmem)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sDone[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sDone[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&sFree[0])), "r"(kTcCons));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&sFree[1])), "r"(kTcCons));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sAbort = 0;
    sArr[0] = sArr[1] = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sTmem;
  const bool producer = warp >= 4;
  const int p = tid - kTcCons;  // producer row
  uint32_t g = 0;               // tiles so far (every role counts alike)
  bool pdead = false;           // producers: a wait of this thread ran out

  for (int it = it0; it < it1; it += istep) {
    const TcItem item = items[it];
    const float c2 = c2v[item.hidx];
    const int ntiles = (item.tot + kTcRows - 1) / kTcRows;
    if (producer) {
      float mloc[DM];  // the query box centre, as the bounds take it
#pragma unroll
      for (int k = 0; k < DM; ++k)
        mloc[k] = k < Q.d ? 0.5f * (Q.lo[(size_t)item.qnode * Q.d + k] + Q.hi[(size_t)item.qnode * Q.d + k]) : 0.f;
      // ---- the item's reference table (warp 4), then the tiles; every
      // producer is past its last read of the previous item's table (the
      // fetches of its tiles) before warp 4 rewrites it
      producers_sync();
      if (warp == 4) {
        int base = 0;
        for (int c0 = 0; c0 < item.ne; c0 += 32) {
          int rb = 0, rn = 0;
          if (c0 + lane < item.ne) {
            const int r = rsorted[item.i0 + c0 + lane] & kNodeMask;
            rb = R.beg[r];
            rn = R.cnt[r];
          }
          int incl = rn;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
          }
          if (c0 + lane < item.ne) {
            sOff[c0 + lane] = base + incl - rn;
            sRb[c0 + lane] = rb;
          }
          base += __shfl_sync(FULL, incl, 31);
        }
      }
      // every producer reaches this barrier once per item; it also decides,
      // for all of them alike, whether to go on after a wait has run out
      if (!producers_sync_and(!pdead && !sAbort)) break;
      const float sw = pow2i(item.a), sr = pow2i(item.b), sbr = pow2i(item.a + item.b - item.s);
      const unsigned norm_a = h2u(__floats2half2_rn(pow2i(item.s), pow2i(item.s)));
      const int ne = item.ne;
      // this thread's reference row of the next tile, loaded one tile ahead
      // so the global reads overlap the tile before (raw: nothing uses the
      // loaded values until the row is staged)
      float4 rv4[DM / 4];
      bool r_ok = false;
      int ent = 0;  // entry of this thread's reference in the last fetched tile
      auto fetch = [&](int tile) {
        const int J = tile * kTcRows + p;
        r_ok = J < item.tot;
        if (r_ok) {
          // the entry holding reference J: a step or two on from the last
          // tile's (references of one entry are consecutive), else a bisection
          int lo = tile == 0 ? 0 : ent, hi = ne;  // sOff[lo] <= J < sOff[hi]
          if (lo + 4 < ne && sOff[lo + 4] <= J) {
            lo += 4;
            while (hi - lo > 1) {
              const int mid = (lo + hi) >> 1;
              if (sOff[mid] <= J) lo = mid; else hi = mid;
            }
          } else {
            while (lo + 1 < ne && sOff[lo + 1] <= J) ++lo;
          }
          ent = lo;
          const float* src = R.pts + (size_t)(sRb[lo] + J - sOff[lo]) * R.dp;
#pragma unroll
          for (int k4 = 0; k4 < DM / 4; ++k4)
            rv4[k4] = 4 * k4 < R.dp ? __ldg(reinterpret_cast<const float4*>(src) + k4) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      };
      for (int qs = 0; qs < item.qn && !pdead; qs += kTcRows) {
        const int qcnt = min(kTcRows, item.qn - qs);
        // A is read by every MMA of the previous block: each producer waits
        // for its last two tiles (a commit tracks only its own thread's
        // MMAs, and the two tiles may have had different issuers; every
        // earlier tile was consumed before these two were staged) before it
        // rewrites its row
        if ((g > 0 && !mbar_wait(&sDone[(g - 1) & 1], ((g - 1) >> 1) & 1u)) ||
            (g > 1 && !mbar_wait(&sDone[g & 1], ((g - 2) >> 1) & 1u))) {
          pdead = true;
          break;
        }
        if (p < qcnt) {
          float v[DM];
#pragma unroll
          for (int k4 = 0; k4 < DM / 4; ++k4) {
            float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * k4 < Q.dp) a4 = __ldg(reinterpret_cast<const float4*>(Q.pts + (size_t)(item.qb + qs + p) * Q.dp) + k4);
            v[4 * k4] = a4.x - mloc[4 * k4];
            v[4 * k4 + 1] = a4.y - mloc[4 * k4 + 1];
            v[4 * k4 + 2] = a4.z - mloc[4 * k4 + 2];
            v[4 * k4 + 3] = a4.w - mloc[4 * k4 + 3];
          }
          unsigned wh[DM / 2], wl[DM / 2];
#pragma unroll
          for (int k = 0; k < DM; k += 2) split2(-2.f * c2 * v[k] * sw, -2.f * c2 * v[k + 1] * sw, wh[k / 2], wl[k / 2]);
          put_row<DM>(tA, p, wh, wh, wl, norm_a);
        } else {
          zero_row<DM>(tA, p);
        }
        fetch(0);
        for (int i = 0; i < ntiles; ++i, ++g) {
          const int b = g & 1;
          // accumulator b and B buffer b are free once the consumers are done
          // with tile g - 2; each producer waits itself before writing its row
          if (g >= 2 && !mbar_wait(&sFree[b], ((g >> 1) - 1) & 1u)) {
            pdead = true;
            break;
          }
          unsigned char* tB = tB0 + b * SH::TILE;
          if (r_ok) {
            float rv[DM];
#pragma unroll
            for (int k4 = 0; k4 < DM / 4; ++k4) {
              rv[4 * k4] = rv4[k4].x - mloc[4 * k4];
              rv[4 * k4 + 1] = rv4[k4].y - mloc[4 * k4 + 1];
              rv[4 * k4 + 2] = rv4[k4].z - mloc[4 * k4 + 2];
              rv[4 * k4 + 3] = rv4[k4].w - mloc[4 * k4 + 3];
            }
            unsigned rh[DM / 2], rl[DM / 2];
#pragma unroll
            for (int k = 0; k < DM; k += 2) split2(rv[k] * sr, rv[k + 1] * sr, rh[k / 2], rl[k / 2]);
            unsigned bn, bl;
            split2(c2 * sumsq<DM>(rv) * sbr, 0.f, bn, bl);
            // norm slots: Bh in the low half, Bl in the high half
            put_row<DM>(tB, p, rh, rl, rh, (bn & 0xffffu) | (bl << 16));
          } else {
            zero_row<DM>(tB, p);
          }
          // the row (and, on the block's first tile, the A row) is handed to
          // the tensor cores' proxy; the producer that stages the tile's last
          // row issues its MMAs, so no producer waits for another
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          if ((atom_add_acq_rel(&sArr[b]) & (kTcRows - 1)) == kTcRows - 1) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_addr(tA), b0 = smem_addr(tB);
            const uint32_t dcol = tmem + (uint32_t)(b * kTcRows);
#pragma unroll
            for (int ks = 0; ks < SH::KC; ++ks) {
              // two K groups (4096 bytes) per K16 step
              const uint64_t ad = tc_desc(a0 + ks * 4096, 2048, 128), bd = tc_desc(b0 + ks * 4096, 2048, 128);
              const uint32_t accum = ks > 0 ? 1u : 0u;
              asm volatile(
                  "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                  "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(accum));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&sDone[b])));
          }
          if (i + 1 < ntiles) fetch(i + 1);
        }
      }
      if (pdead) {
        atomicOr(status, kStTimeout);
        sAbort = 1;
      }
    } else {
      // ---- consumers: row tid of each query block
      const float sout = pow2i(-(item.a + item.b));
      bool ok = true;
      for (int qs = 0; qs < item.qn && ok; qs += kTcRows) {
        const int qcnt = min(kTcRows, item.qn - qs);
        const bool row_ok = tid < qcnt;
        float Aq = 0.f;
        if (row_ok) {
          // A_q = c |q - m|^2 about the query box centre m (as the producers take it)
          float v[DM];
#pragma unroll
          for (int k4 = 0; k4 < DM / 4; ++k4) {
            float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * k4 < Q.dp) a4 = __ldg(reinterpret_cast<const float4*>(Q.pts + (size_t)(item.qb + qs + tid) * Q.dp) + k4);
            v[4 * k4] = a4.x;
            v[4 * k4 + 1] = a4.y;
            v[4 * k4 + 2] = a4.z;
            v[4 * k4 + 3] = a4.w;
          }
#pragma unroll
          for (int k = 0; k < DM; ++k)
            v[k] -= k < Q.d ? 0.5f * (Q.lo[(size_t)item.qnode * Q.d + k] + Q.hi[(size_t)item.qnode * Q.d + k]) : 0.f;
          Aq = c2 * sumsq<DM>(v);
        }
        float acc = 0.f, comp = 0.f;
        for (int i = 0; i < ntiles; ++i, ++g) {
          const int b = g & 1;
          // the warp reads tensor memory together (.sync.aligned): it goes on
          // only if every lane saw the MMA complete
          const bool done = __all_sync(FULL, mbar_wait(&sDone[b], (g >> 1) & 1u));
          if (!done) {
            if (lane == 0) atomicOr(status, kStTimeout);
            sAbort = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int tn = min(kTcRows, item.tot - i * kTcRows);
          const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * kTcRows);
          // 64 columns per step: both 32-column loads in flight together,
          // then two independent chunk sums into one Kahan update
          uint32_t ra[32], rb[32];
          for (int c0 = 0; c0 < tn; c0 += 64) {
            const bool more = c0 + 32 < tn;
            tc_ld32_async(base + c0, ra);
            if (more) tc_ld32_async(base + c0 + 32, rb);
            tc_wait32(ra);
            tc_wait32(rb);
            if (row_ok) {
              float part = ex2_sum32(ra, sout, Aq, tn - c0);
              if (more) part += ex2_sum32(rb, sout, Aq, tn - c0 - 32);
              kahan(acc, comp, part);
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(&sFree[b]);
        }
        if (row_ok && ok) atomicAdd(&gacc[(size_t)item.hidx * Q.n + item.qb + qs + tid], (double)(acc - comp));
      }
      if (!ok) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// The plan buffer: the packed counter and the overflow word (256 bytes kept),
// the items, then one flag per entry.
size_t plan_items_offset() { return 256; }
size_t plan_flags_offset(int n) { return (256 + (size_t)n * sizeof(TcItem) + 255) & ~(size_t)255; }

template <int DM>
void plan_d(const TreeView& Q, const TreeView& R, const TravBuffers& b, const int* rsorted, const int* cnt,
            const int* end, int nkeys, int n, char* base, cudaStream_t s) {
  k_tc_plan<DM><<<(nkeys + 7) / 8, 256, 0, s>>>(
      Q, R, rsorted, cnt, end, nkeys, b.c2, b.inv2h2_up, b.exp_err,
      reinterpret_cast<unsigned char*>(base + plan_flags_offset(n)),
      reinterpret_cast<TcItem*>(base + plan_items_offset()), reinterpret_cast<unsigned long long*>(base), b.base_exp);
}

template <int DM>
cudaError_t sums_d(const TreeView& Q, const TreeView& R, const TravBuffers& b, const int* rsorted, int n,
                   char* base, cudaStream_t s) {
  const int smem = std::max(kTcSmemFloor, TcShape<DM>::SMEM);
  const cudaError_t e = cudaFuncSetAttribute(k_base_tc<DM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  // at most one CTA per item: the count is on the device, so the grid is
  // capped by the entries (an item holds at least one) and the SMs
  // two CTAs per SM fit unless the shared memory takes more than half an SM
  const int per_sm = smem <= 110 * 1024 ? kTcCtasPerSm : 1;
  const int grid = (int)std::min<long>((long)per_sm * b.sms, (long)n);
  k_base_tc<DM><<<grid, kTcThreads, smem, s>>>(Q, R, rsorted, reinterpret_cast<const TcItem*>(base + plan_items_offset()),
                                               reinterpret_cast<const unsigned long long*>(base), b.c2, b.gacc,
                                               b.status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_plan(const TreeView& Q, const TreeView& R, const TravBuffers& b, const int* rsorted,
                           const int* cnt, const int* end, int nkeys, int n, DevBuf& plan,
                           const unsigned char** tcflag, cudaStream_t s, long long* launches) {
  cudaError_t e = plan.ensure(plan_flags_offset(n) + (size_t)n + 256);
  if (e != cudaSuccess) return e;
  char* base = plan.as<char>();
  // the packed counter and the overflow word
  if ((e = cudaMemsetAsync(base, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  if (Q.dp <= 8) plan_d<8>(Q, R, b, rsorted, cnt, end, nkeys, n, base, s);
  else if (Q.dp <= 16) plan_d<16>(Q, R, b, rsorted, cnt, end, nkeys, n, base, s);
  else plan_d<32>(Q, R, b, rsorted, cnt, end, nkeys, n, base, s);
  ++*launches;
  *tcflag = reinterpret_cast<const unsigned char*>(base + plan_flags_offset(n));
  return cudaGetLastError();
}

cudaError_t launch_tc_sums(const TreeView& Q, const TreeView& R, const TravBuffers& b, const int* rsorted, int n,
                           DevBuf& plan, cudaStream_t s, long long* launches) {
  char* base = plan.as<char>();
  cudaError_t e;
  if (Q.dp <= 8) e = sums_d<8>(Q, R, b, rsorted, n, base, s);
  else if (Q.dp <= 16) e = sums_d<16>(Q, R, b, rsorted, n, base, s);
  else e = sums_d<32>(Q, R, b, rsorted, n, base, s);
  ++*launches;
  return e;
}

}  // namespace dfgt
