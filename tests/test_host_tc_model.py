"""The rounding model behind the tensor-core form of the exact sums for
D >= 6 (base_hd_forms.cuh), checked with numpy's float16 on the host: a
float32 value scaled below 2^13 splits into float16 hi + lo with at most
2^-22 of it left over while lo is normal, and the three products
Wh rh + Wh rl + Wl rh miss W r by at most 12u of |W r| (u = 2^-24); an
emulation of the whole form (operands, K layout, K16 steps, the
consumers' fma) stays inside the bound the kernels use."""
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


def pairwise_sumsq(v, dm):
    """|v|^2 as the kernels form it: float32 squares, then pairwise float32
    additions over the padded dimension dm."""
    t = [np.float32(np.float32(x) * np.float32(x)) for x in v] + [np.float32(0.0)] * (dm - len(v))
    while len(t) > 1:
        w = len(t) // 2
        t = [np.float32(t[k] + t[k + w]) for k in range(w)]
    return t[0]


def scales(c2, rho, rmax, f2):
    """The operands' power-of-two scales (hd_tensor_form)."""
    a = 13 - int(np.frexp(2.0 * abs(c2) * rho)[1])
    b = 13 - int(np.frexp(rmax)[1])
    s = int(np.frexp(abs(c2) * f2)[1]) + a + b - 14
    if s > 15:
        x = s - 15
        a -= (x + 1) // 2
        b -= x // 2
        s = 15
    return a, b, max(s, 0)


def emulate_exponent(q, r, m, c2, a, b, s, dm):
    """The tensor form's exponent of one (query, reference) pair, in log2
    units (base_hd_forms.cuh, base_tc.cu), emulated: float32 set-up as on
    the device, float16 splits of W_q 2^a (W_q = -2c q~), r~ 2^b and
    c|r~|^2 2^(a+b-s), exact products summed per K16 step and rounded once
    into the float32 accumulator per step (the model the bound allows 4u
    for), then D 2^-(a+b) + c|q~|^2 with one fma."""
    qt = f32(q - m)
    rt = f32(r - m)
    c2 = np.float32(c2)
    wh, wl = split(f32(f32(np.float32(-2.0) * c2 * qt) * np.float32(2.0 ** a)))
    rh, rl = split(f32(rt * np.float32(2.0 ** b)))
    bn = f32(np.float32(c2 * pairwise_sumsq(rt, dm)) * np.float32(2.0 ** (a + b - s)))
    bh, bl = split(np.array([bn], dtype=np.float32))
    d = len(q)
    pad = lambda v: np.concatenate([v.astype(np.float64), np.zeros(dm - d)])  # noqa: E731
    A = np.concatenate([pad(wh), pad(wh), pad(wl), [2.0 ** s, 2.0 ** s]])
    B = np.concatenate([pad(rh), pad(rl), pad(rh), [float(bh[0]), float(bl[0])]])
    kc = (3 * dm + 2 + 15) // 16
    A = np.concatenate([A, np.zeros(16 * kc - len(A))])
    B = np.concatenate([B, np.zeros(16 * kc - len(B))])
    acc = np.float32(0.0)
    for step in range(kc):
        sl = slice(16 * step, 16 * step + 16)
        acc = np.float32(np.float64(acc) + np.dot(A[sl], B[sl]))
    aq = np.float32(c2 * pairwise_sumsq(qt, dm))
    return float(np.float32(np.float64(acc) * 2.0 ** -(a + b) + np.float64(aq))), kc


def test_bound_covers_the_emulated_form():
    # kappa u |c| (|q~| + |r~|)^2 (log2 units) bounds the exponent's error,
    # kappa = 26 + 4 KC
    rng = np.random.default_rng(4)
    log2e = 1.4426950408889634
    worst = 0.0
    for trial in range(300):
        D = int(rng.choice([6, 8, 12, 16, 20, 32]))
        dm = 8 if D <= 8 else 16 if D <= 16 else 32
        m = f32(rng.random(D))
        rho = float(rng.uniform(0.01, 0.2))
        q = f32(m + rng.uniform(-rho, rho, D) / np.sqrt(D))
        r = f32(m + rng.uniform(-0.5, 0.5, D))
        qt, rt = (q - m).astype(np.float64), (r - m).astype(np.float64)
        for h in (0.05, 0.2, 1.0):
            c2 = float(np.float32(-log2e / (2 * h * h)))
            a, b, s = scales(c2, np.linalg.norm(qt) + 1e-30, np.linalg.norm(rt) + 1e-30, float(rt @ rt) + 1e-30)
            got, kc = emulate_exponent(q, r, m, c2, a, b, s, dm)
            exact = c2 * float(np.sum((q.astype(np.float64) - r.astype(np.float64)) ** 2))
            kappa = 26 + 4 * kc
            bound = kappa * U * abs(c2) * (np.linalg.norm(qt) + np.linalg.norm(rt)) ** 2
            err = abs(got - exact)
            worst = max(worst, err / bound)
            assert err <= bound, (D, h, err, bound)
    assert worst < 0.5  # the emulated accumulation leaves room for the tensor core's own
