"""The rounding model behind the tensor-core form of the exact sums for
D >= 6 (base_hd_forms.cuh), checked with numpy's float16 on the host: a
float32 value scaled below 2^13 splits into float16 hi + lo with at most
2^-22 of it left over while lo is normal, and the three products
Wh rh + Wh rl + Wl rh miss W r by at most 12u of |W r| (u = 2^-24)."""
import numpy as np

U = 2.0 ** -24


def split(v):
    hi = v.astype(np.float16)
    lo = (v - hi.astype(np.float32)).astype(np.float16)
    return hi, lo


def test_split_leaves_at_most_2_pow_minus_22():
    rng = np.random.default_rng(1)
    # magnitudes from 2^-3 (lo still normal) to just below 2^13
    v = (rng.uniform(1.0, 2.0, 200000) * np.exp2(rng.integers(-3, 13, 200000))).astype(np.float32)
    v *= np.where(rng.random(200000) < 0.5, -1, 1).astype(np.float32)
    hi, lo = split(v)
    rest = v.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)
    assert np.all(np.abs(rest) <= 2.0 ** -22 * np.abs(v.astype(np.float64)))
    assert np.all(np.isfinite(hi.astype(np.float32)))


def test_three_products_within_12u():
    rng = np.random.default_rng(2)
    n = 200000
    w = (rng.uniform(-1, 1, n) * np.exp2(rng.integers(-3, 13, n))).astype(np.float32)
    r = (rng.uniform(-1, 1, n) * np.exp2(rng.integers(-3, 13, n))).astype(np.float32)
    keep = (np.abs(w) >= 0.125) & (np.abs(r) >= 0.125)
    w, r = w[keep], r[keep]
    wh, wl = split(w)
    rh, rl = split(r)
    f = lambda a: a.astype(np.float64)  # noqa: E731 -- float16 products are exact in float64
    approx = f(wh) * f(rh) + f(wh) * f(rl) + f(wl) * f(rh)
    exact = f(w) * f(r)
    assert np.all(np.abs(approx - exact) <= 12 * U * np.abs(exact))


def test_subnormal_lo_floor():
    # below 2^-3 the lo part may be subnormal: its error is at most 2^-25
    # absolute, which the form's scales keep 2^-38 below the largest product
    rng = np.random.default_rng(3)
    v = (rng.uniform(1.0, 2.0, 100000) * np.exp2(rng.integers(-20, -3, 100000))).astype(np.float32)
    hi, lo = split(v)
    rest = v.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)
    assert np.all(np.abs(rest) <= 2.0 ** -22 * np.abs(v.astype(np.float64)) + 2.0 ** -25)
