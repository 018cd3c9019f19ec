"""The rounding model behind the tensor-core form of the exact sums for
D >= 6 (base_hd_forms.cuh), checked with numpy's float16 on the host: a
float32 value scaled below 2^13 splits into float16 hi + lo with at most
2^-22 of it left over while lo is normal, and the three products
Wh rh + Wh rl + Wl rh miss W r by at most 12u of |W r| (u = 2^-24); an
emulation of the whole form stays inside the bound the kernels use."""
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


def f32(a):
    return np.asarray(a, dtype=np.float32)


def emulate_exponent(q, r, m, c, a, b):
    """The tensor form's exponent less A_q (base_hd_forms.cuh), emulated:
    float32 set-up as on the device, float16 splits of W 2^a and r~ 2^b,
    exact products, float32 accumulation onto C = B_r 2^(a+b) (the tensor
    core's own accumulation is allowed 8u per step in the bound; plain
    float32 additions stand in for it here), times 2^-(a+b)."""
    qt = f32(q - m)                       # q~, rounded as on the device
    rt = f32(r - m)                       # r~
    w = f32(f32(-2.0 * c) * qt)           # W_q
    b2 = np.float32(0.0)
    for v in rt:                          # B_r = c |r~|^2 by an fma chain
        b2 = np.float32(np.float64(v) * np.float64(v) + np.float64(b2))
    acc = np.float32(np.float32(c) * b2) * np.float32(2.0 ** (a + b))
    wh, wl = split(f32(w * np.float32(2.0 ** a)))
    rh, rl = split(f32(rt * np.float32(2.0 ** b)))
    for k in range(len(q)):
        for x, y in ((wh[k], rh[k]), (wh[k], rl[k]), (wl[k], rh[k])):
            acc = np.float32(np.float64(acc) + np.float64(x) * np.float64(y))
    return np.float64(acc) * 2.0 ** -(a + b)


def test_bound_covers_the_emulated_form():
    # kappa u (|q~| + |r~|)^2 / 2h^2 (natural units) bounds the exponent's
    # error, kappa = max(D+1, 15) + 8 KC; here the set-up and splits are
    # emulated exactly and the accumulation with float32 additions
    rng = np.random.default_rng(4)
    log2e = 1.4426950408889634
    worst = 0.0
    for trial in range(400):
        D = int(rng.choice([6, 8, 12, 16, 20, 32]))
        h = float(np.exp(rng.uniform(np.log(0.05), np.log(1.0))))
        c = -log2e / (2 * h * h)
        m = f32(rng.random(D))
        q = f32(m + rng.uniform(-0.1, 0.1, D))
        r = f32(m + rng.uniform(-0.3, 0.3, D))
        qt, rt = (q - m).astype(np.float64), (r - m).astype(np.float64)
        wmax = 2 * abs(c) * np.linalg.norm(qt) + 1e-30
        rmax = np.linalg.norm(rt) + 1e-30
        a = 13 - int(np.frexp(wmax)[1])
        b = 13 - int(np.frexp(rmax)[1])
        got = emulate_exponent(q, r, m, np.float32(c), a, b)
        exact = c * (np.sum(rt * rt) - 2 * np.dot(qt, rt))
        kc = 3 if D <= 16 else 6  # chained mma steps: DM = 8 or 16 -> 3, DM = 32 -> 6
        kappa = max(D + 1, 15) + 8 * kc
        span2 = (np.linalg.norm(qt) + np.linalg.norm(rt)) ** 2
        bound_log2 = kappa * U * span2 / (2 * h * h) * log2e
        err = abs(got - exact)
        worst = max(worst, err / bound_log2)
        assert err <= bound_log2, (D, h, err, bound_log2)
    assert worst < 0.5  # the emulated accumulation leaves room for the tensor core's own
