// base_hd_forms.cuh -- what the exact-sum kernels (DFGTBase, Section 3.6)
// share: the layout of the sorted base list, and for D >= 6 the choice
// between the direct form (k_base_hd, actions.cu) and the expanded form on
// the tensor cores (k_base_tc, base_tc.cu): both kernels walk the same
// sorted entries and take the same decisions from this code, each summing
// only the runs of its form.
//
// Expanded form about the query box centre m (q~ = q - m, r~ = r - m,
// c = -log2(e)/(2h^2)): x = A_q + B_r + W_q . r~ with A_q = c|q~|^2,
// W_q = -2c q~, B_r = c|r~|^2.  The tensor cores form
// 2^(a+b) (W_q . r~ + B_r) from the float16 splits W_q 2^a = Wh + Wl,
// r~ 2^b = rh + rl (products Wh rh + Wh rl + Wl rh per coordinate) and
// B_r 2^(a+b-s) = Bh + Bl against 2^s, in KC chained K16 steps with a
// float32 accumulator; the result times 2^-(a+b) plus A_q is the exponent.
// The scales bring W_q and r~ just below 2^13 and B_r 2^(a+b-s) below 2^14
// (a and b lowered, at most 8 each, when s would pass 15), so only entries
// well below the largest have subnormal lo parts, whose error (2^-25)
// moves a product by at most 2^-30 of the largest one.
// Rounding, relative to the sum of |terms| <= |c| (|q~| + |r~|)^2:
//   A_q, B_r as pairwise float32 sums of squares, times c: (log2 DM + 2)u <= 7u;
//   q~, r~ and W_q: 3u;
//   the splits: 2^-22 of each operand (4u) twice, and the dropped Wl rl
//   (at most 4u of the product): 12u;  the split of B_r: 4u;
//   each chained K16 step of tcgen05.mma: measured at about 2u of the sum
//   of |terms| (tests/tcgen05_accum_probe.cu), allowed 4u;
// so the exponent is off by at most kappa u |c| (|q~| + |r~|)^2 with
// kappa = 26 + 4 KC.  Since |q~| + |r~| <= 2|q~| + |q - r|, that is at
// most E1 + 2 kappa u |x| with E1 = 8 kappa u |c| rho_Q^2 (rho_Q the radius
// of the query node's points about the box centre): a run takes the tensor form when E1 <= eps_fp / 4 (in
// natural-log units), its scales fit, it has at least kHtMinQ queries and
// holds no self entry (leave-one-out runs take the direct form, which
// leaves the self interaction out exactly).  A term's relative error is
// then at most 2^-21 + eps_fp / 4 + 2 kappa u x, and the float32 row sums
// of positive terms add at most 9u (seven rounding levels per 64-column
// part, Kahan across parts); for the exact sums of a query to stay within
// eps_fp that needs its kernel-weighted mean exponent x~ = sum K x / sum K
// below (3/4 eps_fp - 2^-21 - 9u) / (2 kappa u), as for the direct form's
// (D+4) u x (the self term K = 1 keeps x~ small when Q = R).
#pragma once

#include "common.cuh"

namespace dfgt {
namespace {

// The sorted base list as both kernels read it: warp k takes entries
// [32k, 32k + 32); an entry's reference node sits in the low kNodeBits bits
// of its sorted value, its flags above them.
constexpr int kEntryChunk = 32;
constexpr int kNodeBits = 27;  // node indices stay below 2^27 (checked by the tree build)
constexpr int kNodeMask = (1 << kNodeBits) - 1;

constexpr int kHtMinQ = 16;  // fewer queries leave too many of the 128 tensor rows idle
// chained K16 steps for DM (8, 16 or 32) padded coordinates: three parts
// (Wh rh, Wh rl, Wl rh) of DM slots each and the two slots of B_r
__host__ __device__ constexpr int tc_chunks(int dm) { return ((3 * dm + 2) + 15) / 16; }
constexpr float kHtUnit = 5.9604645e-08f;  // u = 2^-24

// Bounds of a run (query node q against its entries' reference boxes), all
// rounded up: the squared radius of q's points about its box centre (the
// smaller of the box's half diagonal and the node's point radius), and per
// entry the squared distance from that centre to the farthest corner of
// reference box r.
// The query node's part: its box centre (DM slots, zero past d) and rho2.
template <int DM>
__device__ __forceinline__ float hd_query_bounds(const TreeView& Q, int q, float (&mc)[DM]) {
  float rho2 = 0.f;
#pragma unroll
  for (int k = 0; k < DM; ++k) {
    mc[k] = 0.f;
    if (k < Q.d) {
      const float lo = Q.lo[(size_t)q * Q.d + k], hi = Q.hi[(size_t)q * Q.d + k];
      mc[k] = 0.5f * (lo + hi);
      const float w = fmaxf(__fsub_ru(hi, mc[k]), __fsub_ru(mc[k], lo));
      rho2 = __fmaf_ru(w, w, rho2);
    }
  }
  const float rq = Q.rad[q];
  return fminf(rho2, __fmul_ru(rq, rq));
}

// An entry's part: far2 from the query box centre mc.
template <int DM>
__device__ __forceinline__ float hd_entry_far2(const TreeView& R, int r, const float (&mc)[DM]) {
  float far2 = 0.f;
#pragma unroll
  for (int k = 0; k < DM; ++k) {
    if (k < R.d) {
      const float rl = R.lo[(size_t)r * R.d + k], rh = R.hi[(size_t)r * R.d + k];
      const float f = fmaxf(fabsf(__fsub_ru(rh, mc[k])), fabsf(__fsub_rd(rl, mc[k])));
      far2 = __fmaf_ru(f, f, far2);
    }
  }
  return far2;
}

// Scales of a tensor-form run: W_q 2^a, r~ 2^b, B_r 2^(a+b-s) against 2^s.
struct HtScale {
  int a = 0, b = 0, s = 0;
};

// Whether a run takes the tensor form.  d: the dimension; kc: chained K16
// steps; rq2: the query box's squared radius; f2: the largest far2 of the
// run; i2h: 1/(2h^2) rounded up; c2: -log2(e)/(2h^2); qn: the run's queries.
__device__ __forceinline__ bool hd_tensor_form(int d, int kc, float rq2, float f2, float i2h, float c2,
                                               bool self_run, int qn, float exp_err, HtScale* sc) {
  if (self_run || qn < kHtMinQ) return false;
  const float kappa = (float)(26 + 4 * kc);
  (void)d;
  const float e1 = __fmul_ru(__fmul_ru(8.f * kappa * kHtUnit, rq2), i2h);
  if (!(e1 <= exp_err)) return false;
  const float wmax = __fmul_ru(2.f * fabsf(c2), __fsqrt_ru(rq2)), rmax = __fsqrt_ru(f2);
  if (!(rmax > 0.f)) return false;  // every reference at the centre: nothing to expand
  int ew = 0, er = 0, ec = 0;
  if (wmax > 0.f) frexpf(wmax, &ew);  // wmax < 2^ew
  frexpf(rmax, &er);
  frexpf(__fmul_ru(fabsf(c2), f2), &ec);  // |B_r| < 2^ec
  if (ew < -100 || ew > 100 || er < -100 || er > 100 || ec < -100 || ec > 100) return false;
  int a = 13 - ew, b = 13 - er;
  int s = ec + a + b - 14;  // then |B_r| 2^(a+b-s) < 2^14
  if (s > 15) {
    const int x = s - 15;
    if (x > 16) return false;
    a -= (x + 1) / 2;
    b -= x / 2;
    s = 15;
  }
  if (s < 0) s = 0;
  if (a + b > 120 || a + b < -120) return false;
  sc->a = a;
  sc->b = b;
  sc->s = s;
  return true;
}

}  // namespace
}  // namespace dfgt
