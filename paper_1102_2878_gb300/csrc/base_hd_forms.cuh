// base_hd_forms.cuh -- what the exact-sum kernels (DFGTBase, Section 3.6)
// share: the layout of the sorted base list, and for D >= 6 the choice
// between the direct form (k_base_hd, actions.cu) and the expanded form on
// the tensor cores (k_base_hd_tc, base_hd_tc.cu): both kernels walk the
// same sorted entries and take the same decisions from this code, each
// summing only the runs of its form.
//
// Expanded form about the query box centre m (q~ = q - m, r~ = r - m,
// c = -log2(e)/(2h^2)): x = A_q + B_r + W_q . r~ with A_q = c|q~|^2,
// W_q = -2c q~, B_r = c|r~|^2.  The tensor cores sum, per 16 queries x 8
// references, the products Wh rh + Wh rl + Wl rh of the float16 splits
// W_q 2^a = Wh + Wl and r~ 2^b = rh + rl per coordinate onto the C operand
// B_r 2^(a+b), in KC chained mma steps (three parts of DM padded
// coordinates); the result times 2^-(a+b) is the exponent less A_q.  The scales bring both
// operands' largest entries just below 2^13, so only entries below 2^-3
// have subnormal lo parts, whose error (2^-25) moves a product by at most
// 2^-38 of the largest one.
// Rounding, relative to the sum of |terms| <= |c| (|q~| + |r~|)^2:
//   A_q, B_r in float32: (D+1)u each;  q~, r~ and W_q: 3u;
//   the splits: 2^-22 of each operand (4u) twice, and the dropped Wl rl
//   (at most 4u of the product): 12u;
//   each chained mma: measured at up to 4.6u of the sum of |terms| of its
//   inputs (the C operand included), allowed 8u;
// so at most kappa u (|q~| + |r~|)^2 / 2h^2 with kappa = max(D+1, 15) + 8 KC.
// A run takes the tensor form when that is at most E = eps_fp / 4 over the
// query box and the farthest corner of every reference box, it has at
// least kHtMinQ queries and holds no self entry (leave-one-out runs take
// the direct form, which leaves the self interaction out exactly).  A
// term's error is then at most E, within the float allowance eps_fp with
// ex2.approx's 2^-21.
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

constexpr int kHtMinQ = 16;  // the tensor tile is 16 queries high
// chained mma steps for DM (8, 16 or 32) padded coordinates: three parts
// (Wh rh, Wh rl, Wl rh), each one m16n8k8 (DM = 8) or DM/16 m16n8k16
__host__ __device__ constexpr int ht_chunks(int dm) { return dm == 8 ? 3 : 3 * (dm / 16); }
constexpr float kHtUnit = 5.9604645e-08f;  // u = 2^-24

// Squared radius of query box q about its centre and squared distance from
// that centre to the farthest corner of reference box r, rounded up.
__device__ __forceinline__ void hd_entry_bounds(const TreeView& Q, const TreeView& R, int q, int r, float& rho2,
                                                float& far2) {
  rho2 = 0.f;
  far2 = 0.f;
  for (int k = 0; k < Q.d; ++k) {
    const float lo = Q.lo[(size_t)q * Q.d + k], hi = Q.hi[(size_t)q * Q.d + k];
    const float mc = 0.5f * (lo + hi);
    const float w = fmaxf(__fsub_ru(hi, mc), __fsub_ru(mc, lo));
    rho2 = __fmaf_ru(w, w, rho2);
    const float rl = R.lo[(size_t)r * R.d + k], rh = R.hi[(size_t)r * R.d + k];
    const float f = fmaxf(fabsf(__fsub_ru(rh, mc)), fabsf(__fsub_rd(rl, mc)));
    far2 = __fmaf_ru(f, f, far2);
  }
}

// Scales of a tensor-form run: W_q 2^a, r~ 2^b, and 2^-(a+b) on the result.
struct HtScale {
  int a = 0, b = 0;
};

// Whether a run takes the tensor form.  d: the dimension; kc: chained mma
// steps; rq2: the query box's squared radius; f2: the largest far2 of the
// run; i2h: 1/(2h^2) rounded up; c2: -log2(e)/(2h^2); qn: the run's queries.
__device__ __forceinline__ bool hd_tensor_form(int d, int kc, float rq2, float f2, float i2h, float c2,
                                               bool self_run, int qn, float exp_err, HtScale* sc) {
  if (self_run || qn < kHtMinQ) return false;
  const float span = __fadd_ru(__fsqrt_ru(rq2), __fsqrt_ru(f2));
  const float s2 = __fmul_ru(__fmul_ru(span, span), i2h);
  const float kappa = (float)(max(d + 1, 15) + 8 * kc);
  if (!(__fmul_ru(kappa * kHtUnit, s2) <= exp_err)) return false;
  const float wmax = __fmul_ru(2.f * fabsf(c2), __fsqrt_ru(rq2)), rmax = __fsqrt_ru(f2);
  if (!(rmax > 0.f)) return false;  // every reference at the centre: nothing to expand
  int ew = 0, er = 0, ec = 0;
  if (wmax > 0.f) frexpf(wmax, &ew);  // wmax < 2^ew
  frexpf(rmax, &er);
  frexpf(__fmul_ru(fabsf(c2), f2), &ec);  // |B_r| < 2^ec
  if (ew < -100 || ew > 100 || er < -100 || er > 100) return false;
  const int a = 13 - ew, b = 13 - er;
  if (a + b > 120 || a + b < -120 || ec + a + b > 100) return false;
  sc->a = a;
  sc->b = b;
  return true;
}

}  // namespace
}  // namespace dfgt
