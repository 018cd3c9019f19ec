// base_hd_tc.cu -- exact sums (DFGTBase, Section 3.6) for D >= 6 whose
// expanded exponent B_r + W_q . r~ goes through the tensor cores.  The
// form, its error bound and the choice of runs: base_hd_forms.cuh.
//
// One warp per block walks the same 32-entry chunks of the sorted base
// list as k_base_hd and sums the runs (one bandwidth, one query node) that
// take the tensor form; k_base_hd sums the others.  Per run the warp
// stages up to 64 queries as float16 rows (Wh, Wh, Wl per coordinate,
// K = 3D entries padded to 16 KC) and then the references a tile of 64 at
// a time, one lane per reference, as float16 columns (rh, rl, rh) written
// in the order of the mma B fragment (the eight bytes a lane loads for one
// chained step are adjacent), with B_r 2^(a+b) beside them.  Each step of 8
// references runs KC chained m16n8k16 mma per 16 queries; every lane takes
// ex2 of its four results (times 2^-(a+b)) and adds them to the two query
// rows it holds.  Padding references carry C = -1e30 and add 0.
#include <cuda_fp16.h>

#include "base_hd_forms.cuh"
#include "internal.hpp"

namespace dfgt {
namespace {

constexpr int kEntryChunkHt = 32;  // sorted entries per warp (as k_base_hd)
constexpr int kNodeMaskHt = (1 << 27) - 1;
constexpr int kHtQ = 64;           // queries staged at a time
constexpr int kHtTile = 64;        // references per staged tile
constexpr int kHtSteps = kHtTile / 8;
constexpr float kHtPad = -1.0e30f;

template <int DM>
struct HtShape {
  static constexpr int KC = ht_chunks(DM);      // chained k16 steps
  static constexpr int W = 8 * KC;               // 32-bit words of a row or column
};

__device__ __forceinline__ unsigned pack_h2(__half lo, __half hi) {
  return (unsigned)__half_as_ushort(lo) | ((unsigned)__half_as_ushort(hi) << 16);
}

// v = hi + lo + err with |err| <= 2^-22 |v| while lo is normal
__device__ __forceinline__ void split_h(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// 2^e as a float, |e| <= 126
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ void mma16(const unsigned* a, uint2 b, float& d0, float& d1, float& d2, float& d3) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// Kahan step of a float32 running sum.
__device__ __forceinline__ void kahan_add_ht(float& S, float& C, float v) {
  const float y = v - C;
  const float t = S + y;
  C = (t - S) - y;
  S = t;
}

template <int DM>
__global__ void __launch_bounds__(32)
    k_base_hd_tc(TreeView Q, TreeView R, const int* __restrict__ rsorted, const int* __restrict__ ksorted, int n,
                 const float* __restrict__ c2v, const float* __restrict__ inv2h2_up, double* __restrict__ gacc,
                 unsigned long long* __restrict__ tc_ctr, float exp_err) {
  constexpr int KC = HtShape<DM>::KC, W = HtShape<DM>::W;
  // B fragments: step s, chained step c, lane l = 4g + t holds k rows 2t,
  // 2t+1 (x) and 2t+8, 2t+9 (y) of reference column g
  __shared__ __align__(16) uint2 sF[kHtSteps][KC][32];
  __shared__ __align__(16) float sB[kHtTile];
  __shared__ __align__(16) unsigned sQh[kHtQ][W];
  __shared__ float sA[kHtQ];
  __shared__ float2 sAcc[kHtQ];
  __shared__ float sM[DM];
  __shared__ int sOff[2][kEntryChunkHt + 1];
  __shared__ int sRb[2][kEntryChunkHt];
  const int lane = threadIdx.x;
  const long i0 = (long)blockIdx.x * kEntryChunkHt;
  if (i0 >= n) return;
  const int m = (int)min((long)kEntryChunkHt, n - i0);
  const unsigned FULL = 0xffffffffu;
  const int d = Q.d;

  // ---- descriptors, one entry per lane (as k_base_hd)
  int key = -1 - lane, rb = 0, rn = 0, qbeg = 0, qcnt = 0;
  bool self = false;
  float rho2 = 0.f, far2 = 0.f;
  if (lane < m) {
    key = ksorted[i0 + lane];
    const int rv = rsorted[i0 + lane];
    const int r = rv & kNodeMaskHt;
    self = ((rv >> 27) & kSelfFlag) != 0;
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

  // entries past 3D stay zero; rows of padding queries start zero
  for (int i = lane; i < kHtSteps * KC * 32; i += 32) (&sF[0][0][0])[i] = make_uint2(0u, 0u);
  for (int i = lane; i < kHtQ * W; i += 32) (&sQh[0][0])[i] = 0u;
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
      if (!hd_tensor_form(d, KC, rq2, f2, inv2h2_up[hidx], c2r, self_run, qn, exp_err, &sc)) {
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
      // a new query block: rows (Wh, Wh, Wl per coordinate) and A_q
      qcnt_blk = min(kHtQ, qn - qs);
      for (int qi = lane; qi < qcnt_blk; qi += 32) {
        const float* qp = Q.pts + (size_t)(qb + qs + qi) * Q.dp;
        __half hk[16 * KC];
#pragma unroll
        for (int i = 0; i < 16 * KC; ++i) hk[i] = __ushort_as_half((unsigned short)0);
        float a2 = 0.f;
#pragma unroll
        for (int k = 0; k < DM; ++k) {
          if (k < d) {
            const float tqk = __ldg(qp + k) - sM[k];
            a2 = fmaf(tqk, tqk, a2);
            __half hi, lo;
            split_h(-2.f * c2r * tqk * sw, hi, lo);
            hk[3 * k] = hi;
            hk[3 * k + 1] = hi;
            hk[3 * k + 2] = lo;
          }
        }
        uint4* row = reinterpret_cast<uint4*>(&sQh[qi][0]);
#pragma unroll
        for (int v = 0; v < W / 4; ++v)
          row[v] = make_uint4(pack_h2(hk[8 * v], hk[8 * v + 1]), pack_h2(hk[8 * v + 2], hk[8 * v + 3]),
                              pack_h2(hk[8 * v + 4], hk[8 * v + 5]), pack_h2(hk[8 * v + 6], hk[8 * v + 7]));
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
          __half hk[16 * KC];
#pragma unroll
          for (int q = 0; q < 16 * KC; ++q) hk[q] = __ushort_as_half((unsigned short)0);
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
            const float* rp = R.pts + (size_t)(sRb[ts][u] + J - sOff[ts][u]) * R.dp;
            float b2 = 0.f;
#pragma unroll
            for (int k = 0; k < DM; ++k) {
              if (k < d) {
                const float rk = __ldg(rp + k) - sM[k];
                b2 = fmaf(rk, rk, b2);
                __half hi, lo;
                split_h(rk * sr, hi, lo);
                hk[3 * k] = hi;
                hk[3 * k + 1] = lo;
                hk[3 * k + 2] = hi;
              }
            }
            cb = c2r * b2 * sc_c;
          }
          // chained step c, pair p of the column: lane 4g + (p mod 4), x for p < 4
#pragma unroll
          for (int c = 0; c < KC; ++c) {
            uint4* col = reinterpret_cast<uint4*>(&sF[j >> 3][c][(j & 7) * 4]);
            const __half* h = hk + 16 * c;
            col[0] = make_uint4(pack_h2(h[0], h[1]), pack_h2(h[8], h[9]), pack_h2(h[2], h[3]), pack_h2(h[10], h[11]));
            col[1] = make_uint4(pack_h2(h[4], h[5]), pack_h2(h[12], h[13]), pack_h2(h[6], h[7]), pack_h2(h[14], h[15]));
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
    for (int q0 = 0; q0 < qcnt_blk; q0 += 16) {
      unsigned a[KC][4];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        a[c][0] = sQh[q0 + g][8 * c + tq];
        a[c][1] = sQh[q0 + g + 8][8 * c + tq];
        a[c][2] = sQh[q0 + g][8 * c + tq + 4];
        a[c][3] = sQh[q0 + g + 8][8 * c + tq + 4];
      }
      const float2* B2 = reinterpret_cast<const float2*>(&sB[0]) + tq;
      float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int st = 0; st < nst; ++st) {
        const float2 bc = B2[st * 4];
        float d0 = bc.x, d1 = bc.y, d2 = bc.x, d3 = bc.y;
#pragma unroll
        for (int c = 0; c < KC; ++c) mma16(a[c], sF[st][c][lane], d0, d1, d2, d3);
        const float2 xa = __fmul2_rn(make_float2(d0, d2), so2), xb = __fmul2_rn(make_float2(d1, d3), so2);
        pa = __fadd2_rn(pa, make_float2(ex2_approx(xa.x), ex2_approx(xa.y)));
        pb = __fadd2_rn(pb, make_float2(ex2_approx(xb.x), ex2_approx(xb.y)));
      }
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
  const int grid = (int)((n + kEntryChunkHt - 1) / kEntryChunkHt);
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
