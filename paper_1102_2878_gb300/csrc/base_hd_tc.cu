// base_hd_tc.cu -- exact sums (DFGTBase, Section 3.6) for D >= 6 whose
// expanded exponent B_r + W_q . r~ goes through the tensor cores.  The
// form, its error bound and the choice of runs: base_hd_forms.cuh.
//
// One warp per block walks the same 32-entry chunks of the sorted base
// list as k_base_hd and sums the runs (one bandwidth, one query node) that
// take the tensor form; k_base_hd sums the others.  The contraction is
// split by parts: Wh . rh + Wh . rl + Wl . rh, each a dot product over the
// DM (padded) coordinates, so a query row stores Wh and Wl (DM float16
// each) and a reference column rh and rl, both converted two coordinates
// at a time.  Per run the warp stages up to 64 queries, then the
// references a tile of 64 at a time, one lane per reference, written in
// the order of the mma B fragment (the bytes a lane loads for one step are
// adjacent), with B_r 2^(a+b) beside them.  Each step of 8 references runs
// 3 DM/16 chained m16n8k16 mma (3 m16n8k8 for DM = 8) per 16 queries;
// every lane takes ex2 of its four results (times 2^-(a+b)) and adds them
// to the two query rows it holds.  Padding references carry C = -1e30 and
// add 0.
#include <cuda_fp16.h>

#include "base_hd_forms.cuh"
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kHtQ = 64;           // queries staged at a time
constexpr int kHtTile = 128;       // references per staged tile
constexpr int kHtSteps = kHtTile / 8;
constexpr float kHtPad = -1.0e30f;

template <int DM>
struct HtShape {
  static constexpr bool K8 = DM == 8;            // m16n8k8 steps, else m16n8k16
  static constexpr int NCH = K8 ? 1 : DM / 16;   // mma steps per part
  static constexpr int HW = DM / 2;              // 32-bit words of one part (DM float16)
  static constexpr int KW = K8 ? 4 : 8;          // words of one step's column
  static_assert(DM == 8 || DM == 16 || DM == 32, "DM is 8, 16 or 32");
  static_assert(3 * NCH == ht_chunks(DM), "the chained steps of the error bound");
};

__device__ __forceinline__ unsigned h2_bits(__half2 h) {
  unsigned u;
  memcpy(&u, &h, sizeof u);
  return u;
}

// (v.x, v.y) = hi + lo + err per element, |err| <= 2^-22 |v| while lo is normal
__device__ __forceinline__ void split_h2(float2 v, unsigned& hi, unsigned& lo) {
  const __half2 h = __float22half2_rn(v);
  const float2 b = __half22float2(h);
  hi = h2_bits(h);
  lo = h2_bits(__float22half2_rn(make_float2(v.x - b.x, v.y - b.y)));
}

// 2^e as a float, |e| <= 126
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ void mma16(const unsigned* a, uint2 b, float& d0, float& d1, float& d2, float& d3) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ void mma8(const unsigned* a, unsigned b, float& d0, float& d1, float& d2, float& d3) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a[0]), "r"(a[1]), "r"(b));
}

// Kahan step of a float32 running sum.
__device__ __forceinline__ void kahan_add_ht(float& S, float& C, float v) {
  const float y = v - C;
  const float t = S + y;
  C = (t - S) - y;
  S = t;
}

// DM coordinates of a tree row (dp floats, zero-padded, 16-byte aligned) minus the centre
template <int DM>
__device__ __forceinline__ void load_centred(const float* __restrict__ p, int dp, const float* __restrict__ m,
                                             float* v) {
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

template <int DM>
__global__ void __launch_bounds__(32)
    k_base_hd_tc(TreeView Q, TreeView R, const int* __restrict__ rsorted, const int* __restrict__ ksorted, int n,
                 const float* __restrict__ c2v, const float* __restrict__ inv2h2_up, double* __restrict__ gacc,
                 unsigned long long* __restrict__ tc_ctr, float exp_err) {
  using SH = HtShape<DM>;
  constexpr int NCH = SH::NCH, HW = SH::HW, KW = SH::KW;
  // B fragments: step s, part (rh, rl), mma step c, then the words of lane
  // l = 4g + t: k rows 2t, 2t+1 (and 2t+8, 2t+9 for k16) of reference column g
  __shared__ __align__(16) unsigned sF[kHtSteps][2][NCH][32 * KW / 4];
  __shared__ __align__(16) float sB[kHtTile];
  // query rows: Wh, then Wl, then 4 words of padding (the A-fragment loads
  // of the 8 rows g then fall on distinct banks)
  __shared__ __align__(16) unsigned sQh[kHtQ][2 * HW + 4];
  __shared__ float sA[kHtQ];
  __shared__ float2 sAcc[kHtQ];
  __shared__ float sM[DM];
  __shared__ int sOff[2][kEntryChunk + 1];
  __shared__ int sRb[2][kEntryChunk];
  const int lane = threadIdx.x;
  const long i0 = (long)blockIdx.x * kEntryChunk;
  if (i0 >= n) return;
  const int m = (int)min((long)kEntryChunk, n - i0);
  const unsigned FULL = 0xffffffffu;
  const int d = Q.d;

  // ---- descriptors, one entry per lane (as k_base_hd)
  int key = -1 - lane, rb = 0, rn = 0, qbeg = 0, qcnt = 0;
  bool self = false;
  float rho2 = 0.f, far2 = 0.f;
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
    hd_entry_bounds(Q, R, q, r, rho2, far2);
  }
  const int keyp = __shfl_up_sync(FULL, key, 1);
  const unsigned starts = __ballot_sync(FULL, lane < m && (lane == 0 || key != keyp));
  auto run_end = [&](int t) -> int {
    const unsigned later = starts & ~((2u << t) - 1u);
    return later ? __ffs(later) - 1 : m;
  };
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
      sOff[sl][lane - t] = incl - in_run;
      sRb[sl][lane - t] = rb;
    }
    if (lane == 0) sOff[sl][e - t] = tot;
    __syncwarp();
    return tot;
  };

  // rows of padding queries start zero (their sums are dropped)
  for (int i = lane; i < kHtQ * (2 * HW + 4); i += 32) (&sQh[0][0])[i] = 0u;
  __syncwarp();

  int t = 0, e = run_end(0), ts = 0, qs = 0, j0 = 0;
  int tot = build_table(t, e, ts);
  float c2r = 0.f, sw = 1.f, sr = 1.f, sout = 1.f, sc_c = 1.f;
  int qb = 0, qn = 0, hidx = 0, qcnt_blk = 0;
  bool new_run = true;
  const int g = lane >> 2, tq = lane & 3;
  while (true) {
    if (new_run) {
      const int key_t = __shfl_sync(FULL, key, t);
      hidx = key_t / Q.nn;
      const int qnode = key_t - hidx * Q.nn;
      c2r = c2v[hidx];
      qb = __shfl_sync(FULL, qbeg, t);
      qn = __shfl_sync(FULL, qcnt, t);
      const float rq2 = __shfl_sync(FULL, rho2, t);
      const float f2 = __uint_as_float(
          __reduce_max_sync(FULL, (lane >= t && lane < e) ? __float_as_uint(far2) : 0u));
      const bool self_run = __any_sync(FULL, lane >= t && lane < e && self);
      HtScale sc;
      if (!hd_tensor_form(d, ht_chunks(DM), rq2, f2, inv2h2_up[hidx], c2r, self_run, qn, exp_err, &sc)) {
        // summed by k_base_hd: on to the next run
        if (e >= m) break;
        t = e;
        e = run_end(t);
        ts ^= 1;
        tot = build_table(t, e, ts);
        continue;
      }
      sw = pow2f(sc.a);
      sr = pow2f(sc.b);
      sc_c = pow2f(sc.a + sc.b);
      sout = pow2f(-(sc.a + sc.b));
      // the query box centre, as the traversal's bounds take it
      for (int k = lane; k < DM; k += 32)
        sM[k] = k < d ? 0.5f * (Q.lo[(size_t)qnode * d + k] + Q.hi[(size_t)qnode * d + k]) : 0.f;
      if (lane == 0) atomicAdd(tc_ctr, (unsigned long long)qn * tot);
      __syncwarp();
      new_run = false;
    }
    if (j0 == 0) {
      // a new query block: rows Wh then Wl (DM float16 each) and A_q
      qcnt_blk = min(kHtQ, qn - qs);
      for (int qi = lane; qi < qcnt_blk; qi += 32) {
        float v[DM];
        load_centred<DM>(Q.pts + (size_t)(qb + qs + qi) * Q.dp, Q.dp, sM, v);
        float a2 = 0.f;
        unsigned wh[HW], wl[HW];
#pragma unroll
        for (int k = 0; k < DM; k += 2) {
          a2 = fmaf(v[k], v[k], a2);
          a2 = fmaf(v[k + 1], v[k + 1], a2);
          split_h2(make_float2(-2.f * c2r * v[k] * sw, -2.f * c2r * v[k + 1] * sw), wh[k / 2], wl[k / 2]);
        }
        uint4* row = reinterpret_cast<uint4*>(&sQh[qi][0]);
#pragma unroll
        for (int w = 0; w < HW / 4; ++w) {
          row[w] = make_uint4(wh[4 * w], wh[4 * w + 1], wh[4 * w + 2], wh[4 * w + 3]);
          row[HW / 4 + w] = make_uint4(wl[4 * w], wl[4 * w + 1], wl[4 * w + 2], wl[4 * w + 3]);
        }
        sA[qi] = c2r * a2;
        sAcc[qi] = make_float2(0.f, 0.f);
      }
    }
    const int tn = min(kHtTile, tot - j0);
    const int nst = (tn + 7) >> 3;
    {
      // references [j0, j0 + tn) of the run, lane per reference
      int u = -1;
#pragma unroll
      for (int i = 0; i < kHtTile / 32; ++i) {
        const int j = lane + 32 * i;
        if (j < nst * 8) {
          unsigned rh[HW], rl[HW];
#pragma unroll
          for (int w = 0; w < HW; ++w) rh[w] = rl[w] = 0u;
          float cb = kHtPad;
          if (j < tn) {
            const int J = j0 + j;
            if (u < 0) {
              int lo = 0, hi = e - t;  // sOff[lo] <= J < sOff[hi]
              while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (sOff[ts][mid] <= J) lo = mid; else hi = mid;
              }
              u = lo;
            } else {
              while (sOff[ts][u + 1] <= J) ++u;
            }
            float v[DM];
            load_centred<DM>(R.pts + (size_t)(sRb[ts][u] + J - sOff[ts][u]) * R.dp, R.dp, sM, v);
            float b2 = 0.f;
#pragma unroll
            for (int k = 0; k < DM; k += 2) {
              b2 = fmaf(v[k], v[k], b2);
              b2 = fmaf(v[k + 1], v[k + 1], b2);
              split_h2(make_float2(v[k] * sr, v[k + 1] * sr), rh[k / 2], rl[k / 2]);
            }
            cb = c2r * b2 * sc_c;
          }
          // part p, mma step c: the column's KW words go to lanes 4g .. 4g+3
          // (k16: lane t takes words t and t+4); the two 16-byte halves are
          // written in an order that spreads the warp over the banks
          const int g8 = j & 7, flip = (g8 >> 2) & 1;
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const unsigned* w = p == 0 ? rh : rl;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
              uint4* col = reinterpret_cast<uint4*>(&sF[j >> 3][p][c][g8 * KW]);
              const unsigned* x = w + KW * c;
              if constexpr (SH::K8) {
                col[0] = make_uint4(x[0], x[1], x[2], x[3]);
              } else {
                const uint4 h0 = make_uint4(x[0], x[4], x[1], x[5]), h1 = make_uint4(x[2], x[6], x[3], x[7]);
                col[flip] = flip ? h1 : h0;
                col[flip ^ 1] = flip ? h0 : h1;
              }
            }
          }
          sB[j] = cb;
        }
      }
    }
    __syncwarp();
    // the next segment: next tile, else next query block, else next run
    int nt = t, ne = e, nts = ts, nqs = qs, nj0 = j0 + kHtTile, ntot = tot;
    const bool last_tile = nj0 >= tot;
    if (last_tile) {
      nj0 = 0;
      nqs = qs + kHtQ;
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

    // this tile against the block's queries, 16 at a time
    const float2 so2 = make_float2(sout, sout);
    auto load_a = [&](int q0, unsigned (&ah)[NCH][4], unsigned (&al)[NCH][4]) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        ah[c][0] = sQh[q0 + g][KW * c + tq];
        ah[c][1] = sQh[q0 + g + 8][KW * c + tq];
        al[c][0] = sQh[q0 + g][HW + KW * c + tq];
        al[c][1] = sQh[q0 + g + 8][HW + KW * c + tq];
        if constexpr (!SH::K8) {
          ah[c][2] = sQh[q0 + g][KW * c + tq + 4];
          ah[c][3] = sQh[q0 + g + 8][KW * c + tq + 4];
          al[c][2] = sQh[q0 + g][HW + KW * c + tq + 4];
          al[c][3] = sQh[q0 + g + 8][HW + KW * c + tq + 4];
        }
      }
    };
    // the exponents of one step for the 16 rows held in ah, al: Wh rh + Wh rl + Wl rh onto C
    auto step = [&](const unsigned (&ah)[NCH][4], const unsigned (&al)[NCH][4], int st, float2 bc,
                    float2& pa, float2& pb) {
      float d0 = bc.x, d1 = bc.y, d2 = bc.x, d3 = bc.y;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        if constexpr (SH::K8) {
          const unsigned bh = sF[st][0][c][lane], bl = sF[st][1][c][lane];
          mma8(ah[c], bh, d0, d1, d2, d3);
          mma8(ah[c], bl, d0, d1, d2, d3);
          mma8(al[c], bh, d0, d1, d2, d3);
        } else {
          const uint2 bh = reinterpret_cast<const uint2*>(sF[st][0][c])[lane];
          const uint2 bl = reinterpret_cast<const uint2*>(sF[st][1][c])[lane];
          mma16(ah[c], bh, d0, d1, d2, d3);
          mma16(ah[c], bl, d0, d1, d2, d3);
          mma16(al[c], bh, d0, d1, d2, d3);
        }
      }
      const float2 xa = __fmul2_rn(make_float2(d0, d2), so2), xb = __fmul2_rn(make_float2(d1, d3), so2);
      pa = __fadd2_rn(pa, make_float2(ex2_approx(xa.x), ex2_approx(xa.y)));
      pb = __fadd2_rn(pb, make_float2(ex2_approx(xb.x), ex2_approx(xb.y)));
    };
    auto row_sums = [&](int q0, float2 pa, float2 pb) {
      float vg = pa.x + pb.x, vh = pa.y + pb.y;  // rows q0 + g and q0 + g + 8
      vg += __shfl_xor_sync(FULL, vg, 1);
      vh += __shfl_xor_sync(FULL, vh, 1);
      vg += __shfl_xor_sync(FULL, vg, 2);
      vh += __shfl_xor_sync(FULL, vh, 2);
      if (tq == 0) {
        if (q0 + g < qcnt_blk) {
          float2 acc = sAcc[q0 + g];
          kahan_add_ht(acc.x, acc.y, vg);
          sAcc[q0 + g] = acc;
        }
        if (q0 + g + 8 < qcnt_blk) {
          float2 acc = sAcc[q0 + g + 8];
          kahan_add_ht(acc.x, acc.y, vh);
          sAcc[q0 + g + 8] = acc;
        }
      }
    };
    const float2* B2 = reinterpret_cast<const float2*>(&sB[0]) + tq;
    int q0 = 0;
    if constexpr (DM <= 16) {
      // 32 queries a sweep: two row blocks share each step's B fragments
      for (; q0 + 16 < qcnt_blk; q0 += 32) {
        unsigned ah[NCH][4], al[NCH][4], eh[NCH][4], el[NCH][4];
        load_a(q0, ah, al);
        load_a(q0 + 16, eh, el);
        float2 pa = make_float2(0.f, 0.f), pb = pa, ra = pa, rb2 = pa;
#pragma unroll 2
        for (int st = 0; st < nst; ++st) {
          const float2 bc = B2[st * 4];
          step(ah, al, st, bc, pa, pb);
          step(eh, el, st, bc, ra, rb2);
        }
        row_sums(q0, pa, pb);
        row_sums(q0 + 16, ra, rb2);
      }
    }
    for (; q0 < qcnt_blk; q0 += 16) {
      unsigned ah[NCH][4], al[NCH][4];
      load_a(q0, ah, al);
      float2 pa = make_float2(0.f, 0.f), pb = pa;
#pragma unroll 2
      for (int st = 0; st < nst; ++st) step(ah, al, st, B2[st * 4], pa, pb);
      row_sums(q0, pa, pb);
    }
    if (last_tile) {
      // the block's sums, scaled by 2^A_q, one atomic per query
      __syncwarp();
      for (int qi = lane; qi < qcnt_blk; qi += 32) {
        const float2 acc = sAcc[qi];
        const float v = (acc.x - acc.y) * exp2f(sA[qi]);
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

}  // namespace

cudaError_t launch_base_hd_tc(const TreeView& Q, const TreeView& R, const TravBuffers& b, const int* rsorted,
                              const int* ksorted, int n, cudaStream_t s, long long* launches) {
  if (n <= 0 || Q.d < 6) return cudaSuccess;
  const int grid = (int)((n + kEntryChunk - 1) / kEntryChunk);
  if (Q.dp <= 8)
    k_base_hd_tc<8><<<grid, 32, 0, s>>>(Q, R, rsorted, ksorted, n, b.c2, b.inv2h2_up, b.gacc, b.base_exp, b.exp_err);
  else if (Q.dp <= 16)
    k_base_hd_tc<16><<<grid, 32, 0, s>>>(Q, R, rsorted, ksorted, n, b.c2, b.inv2h2_up, b.gacc, b.base_exp, b.exp_err);
  else
    k_base_hd_tc<32><<<grid, 32, 0, s>>>(Q, R, rsorted, ksorted, n, b.c2, b.inv2h2_up, b.gacc, b.base_exp, b.exp_err);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace dfgt
