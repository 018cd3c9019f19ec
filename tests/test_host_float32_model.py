"""The rounding models behind the float32 exponents of the exact sums, checked
by emulating the kernels' float32 operations on the host.  The expanded form
of the D <= 5 sums is described at its tests below.  The direct form (the
brute force, the D <= 5 exact sums in direct form and the D >= 6 SIMT exact
sums all compute a term the same way): D float32 differences q_k - r_k,
their squares summed by a chain of fused multiply-adds, one float32 product
with c = fl(-log2(e) / (2h^2)), then 2^x.  Counting first-order relative
errors of the exponent x = |q - r|^2 / (2h^2) (u = 2^-24): 2u from squaring
a rounded difference, one u per fused multiply-add of the chain (D, the
first included), u for c and u for the product, so (D+4) u x of relative
error per term; the GPU parity tests allow that plus 2^-21 for ex2.approx.
These tests emulate the float32 operations in the kernels' order on the
host, with a correctly rounded fused multiply-add, take 2^x exactly so that
only the exponent's rounding is measured, check the allowance against
float64 exp(-x), and keep one input on which an allowance of (D+3) u x
fails."""
import numpy as np
import pytest

U = 2.0 ** -24
LOG2E = 1.4426950408889634
f32, f64 = np.float32, np.float64


def fma32(a, b, c):
    """Correctly rounded float32 a*b + c: the float64 product of two float32
    values is exact, TwoSum gives p + c as hi + lo exactly, and hi rounded to
    float32 is corrected where it sits exactly halfway between two float32
    values and lo decides the direction."""
    p = a.astype(f64) * b.astype(f64)
    c = c.astype(f64)
    hi = p + c
    bb = hi - p
    lo = (p - (hi - bb)) + (c - bb)
    r = hi.astype(f32)
    rd = r.astype(f64)
    up = np.nextafter(r, f32(np.inf)).astype(f64)
    dn = np.nextafter(r, f32(-np.inf)).astype(f64)
    # hi exactly halfway between r and a neighbour, and lo pulling away from r
    tie_up = (hi == (rd + up) / 2) & (lo > 0)
    tie_dn = (hi == (rd + dn) / 2) & (lo < 0)
    r = np.where(tie_up, up.astype(f32), r)
    r = np.where(tie_dn, dn.astype(f32), r)
    # (in the other tie cases lo pulls towards r, which is then right)
    return r.astype(f32)


def kernel_exponent(q, r, h):
    """x as the kernels compute it: float32 differences, a fused multiply-add
    chain over the coordinates in order, one product with float32 c."""
    inv = 1.0 / (2.0 * h * h)
    c = f32(-LOG2E * inv)  # one rounding of a float64 value, as the library does
    d2 = np.zeros(q.shape[0], dtype=f32)
    for k in range(q.shape[1]):
        t = (q[:, k] - r[:, k]).astype(f32)  # float32 subtraction, one rounding
        d2 = fma32(t, t, d2)
    return (d2 * c).astype(f32)


def check(q, r, h):
    """Largest ratio of the emulated term's relative error to (D+4) u x."""
    D = q.shape[1]
    x = ((q.astype(f64) - r.astype(f64)) ** 2).sum(1) / (2.0 * h * h)
    term = np.exp2(kernel_exponent(q, r, h).astype(f64))
    K = np.exp(-x)
    rel = np.abs(term / K - 1.0)
    allow = (D + 4) * U * x
    # second-order terms: e^(x theta) - 1 <= x theta (1 + x theta), with
    # x theta < 1e-3 here, inside the 1e-3 slack below
    assert np.all(allow < 1e-3)
    assert np.all(rel <= allow * (1.0 + 1e-3) + 1e-15), float((rel / np.maximum(allow, 1e-300)).max())
    ok = allow > 0
    return float((rel[ok] / allow[ok]).max()) if ok.any() else 0.0


def test_fma32_is_correctly_rounded():
    # against exact rational arithmetic on a sample, ties included
    from fractions import Fraction

    rng = np.random.default_rng(3)
    a = rng.standard_normal(4000).astype(f32)
    c = (rng.standard_normal(4000) * np.exp2(rng.integers(-30, 10, 4000))).astype(f32)
    # constructed ties: a*a + c exactly halfway between two float32 values
    # before lo, with c tiny so that lo decides
    a[:8] = f32(1.0) + f32(2.0 ** -12)   # a^2 = 1 + 2^-11 + 2^-24: halfway above 1 + 2^-11
    c[:4] = f32(2.0 ** -60)
    c[4:8] = f32(-(2.0 ** -60))
    got = fma32(a, a, c)
    for i in range(len(a)):
        exact = Fraction(float(a[i])) * Fraction(float(a[i])) + Fraction(float(c[i]))
        g = Fraction(float(got[i]))
        lo = Fraction(float(np.nextafter(got[i], f32(-np.inf))))
        hi = Fraction(float(np.nextafter(got[i], f32(np.inf))))
        # nearest: no float32 neighbour is closer to the exact value
        assert abs(g - exact) <= abs(lo - exact) and abs(g - exact) <= abs(hi - exact), i
    assert got[0] == np.nextafter(f32(1.0 + 2.0 ** -11), f32(2.0))  # lo > 0 rounds up
    assert got[4] == f32(1.0 + 2.0 ** -11)                          # lo < 0 rounds down


@pytest.mark.parametrize("D", [1, 2, 3, 5, 8, 16, 32])
def test_random_terms_within_allowance(D):
    rng = np.random.default_rng(10 + D)
    n = 20000
    q = rng.random((n, D)).astype(f32)
    r = rng.random((n, D)).astype(f32)
    # bandwidths that put x = |q - r|^2 / 2h^2 between about 0 and 80
    dist2 = ((q.astype(f64) - r.astype(f64)) ** 2).sum(1)
    worst = 0.0
    for xt in (0.05, 1.0, 10.0, 40.0, 80.0):
        h = float(np.sqrt(np.median(dist2) / (2.0 * xt)))
        sel = dist2 / (2 * h * h) <= 80.0
        worst = max(worst, check(q[sel], r[sel], h))
    # random terms reach a visible part of the allowance (0.77 of it at D = 1,
    # 0.16 at D = 32)
    assert 0.1 < worst <= 1.0 + 1e-3, worst


def test_one_u_less_is_not_enough():
    # D = 1: a difference just above 1 that rounds by nearly half an ulp, and
    # a bandwidth whose float32 c is rounded by nearly u; the term's error is
    # 4.89 u x, above (D+3) u x = 4 u x and within (D+4) u x
    q = np.array([[float.fromhex("0x1.03950ap+0")]], dtype=f32)
    r = np.array([[float.fromhex("0x1.fdcp-25")]], dtype=f32)
    h = 1.1997795487517997
    ratio = check(q, r, h)  # against (D+4) u x
    assert 4.0 / 5.0 < ratio <= 1.0, ratio


@pytest.mark.parametrize("D", [3, 16, 32])
def test_adversarial_terms_within_allowance(D):
    # the differences rounded (q just above 1, r a multiple of 2^-25 below
    # 2^-15: q - r needs a bit below float32's last one whenever r is an odd
    # multiple) and all D coordinates alike, so the chain adds equal squares
    # and its roundings tend the same way
    rng = np.random.default_rng(100 + D)
    n = 20000
    base = f32(1.0) + (rng.integers(1, 2 ** 20, (n, 1)) * 2.0 ** -23).astype(f32)
    q = np.repeat(base, D, axis=1).astype(f32)
    r = (rng.integers(1, 2 ** 10, (n, 1)) * 2.0 ** -25 + 2.0 ** -25).astype(f32)
    r = np.repeat(r, D, axis=1).astype(f32)
    dist2 = ((q.astype(f64) - r.astype(f64)) ** 2).sum(1)
    for xt in (1.0, 30.0, 80.0):
        h = float(np.sqrt(dist2.max() / (2.0 * xt)))
        check(q, r, h)


def test_coincident_points_give_one():
    q = np.random.default_rng(5).random((100, 16)).astype(f32)
    assert np.all(kernel_exponent(q, q, 0.3) == 0.0)
    assert check(q, q, 0.3) == 0.0


def test_emulation_rounds_every_step():
    # the emulated exponent is further from the exact one than a single
    # float32 rounding of it: the emulation does round each step in float32
    # (an emulation that kept float64 intermediates would pass the allowance
    # checks trivially)
    rng = np.random.default_rng(8)
    q = rng.random((5000, 16)).astype(f32)
    r = rng.random((5000, 16)).astype(f32)
    h = 0.3
    x = ((q.astype(f64) - r.astype(f64)) ** 2).sum(1) * (-LOG2E / (2 * h * h))
    once = np.abs(x.astype(f32).astype(f64) - x)
    emul = np.abs(kernel_exponent(q, r, h).astype(f64) - x)
    assert emul.mean() > 2 * once.mean()


# ---- the expanded form (D <= 5 exact sums) ----
#
# About the query box centre m, with q~ = q - m and r~ = r - m rounded in
# float32: A_q = fl(c |q~|^2) and B_r = fl(c |r~|^2) from fused multiply-add
# chains, W_q = fl(-2c q~), and S = B_r + W_q . r~ by a chain of D fused
# multiply-adds that starts from B_r; the exponent is A_q + S (2^S is summed
# and the sum scaled by 2^A_q, so A_q + S is never rounded).  Its error,
# in natural units, is at most u ((D+4) (|q~| + |r~|)^2 + D |r~|^2) / 2h^2.


def expanded_exponent(q, r, m, h):
    """A_q + S (log2 units, float64 sum of the two float32 values) and the
    rounded offsets q~, r~, in the kernel's operation order."""
    inv = 1.0 / (2.0 * h * h)
    c = f32(-LOG2E * inv)
    n, D = q.shape
    qt = (q - m).astype(f32)
    rt = (r - m).astype(f32)
    a2 = np.zeros(n, f32)
    b2 = np.zeros(n, f32)
    for k in range(D):
        a2 = fma32(qt[:, k], qt[:, k], a2)
        b2 = fma32(rt[:, k], rt[:, k], b2)
    A = (c * a2).astype(f32)
    B = (c * b2).astype(f32)
    W = ((f32(-2.0) * c) * qt).astype(f32)  # -2c is exact; one rounding
    S = B
    for k in range(D):
        S = fma32(W[:, k], rt[:, k], S)
    return A.astype(f64) + S.astype(f64), qt, rt


def expanded_ratios(q, r, m, h):
    """The exponent's error (natural units) over the corrected bound and over
    (D+4) u (|q~| + |r~|)^2 / 2h^2 alone."""
    D = q.shape[1]
    xh, qt, rt = expanded_exponent(q, r, m, h)
    xe = -LOG2E * ((q.astype(f64) - r.astype(f64)) ** 2).sum(1) / (2 * h * h)
    err = np.abs(xh - xe) / LOG2E
    nq = np.sqrt((qt.astype(f64) ** 2).sum(1))
    nr = np.sqrt((rt.astype(f64) ** 2).sum(1))
    old = (D + 4) * U * (nq + nr) ** 2 / (2 * h * h)
    new = old + D * U * nr ** 2 / (2 * h * h)
    return err / new, err / old


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5])
def test_expanded_exponent_within_bound(D):
    rng = np.random.default_rng(200 + D)
    n = 50000
    worst = 0.0
    for side, h in ((1.0, 0.3), (0.1, 0.05), (0.01, 0.02)):
        # a query box of the given side about its centre, references anywhere
        m = rng.random((1, D)).astype(f32)
        q = (m + side * (rng.random((n, D)) - 0.5)).astype(f32)
        r = rng.random((n, D)).astype(f32)
        rn, _ = expanded_ratios(q, r, m, h)
        worst = max(worst, float(rn.max()))
    assert worst <= 1.0 + 1e-3, worst


def test_chain_from_b_r_breaks_the_bound_without_its_term():
    # D = 5, m = 0: |B_r| just above a power of two and every W_k r~_k just
    # under half an ulp of it, so each step of the chain rounds its addend
    # away in the same direction; the error exceeds (D+4) u (|q~| + |r~|)^2 /
    # 2h^2 and stays within the bound with the D |r~|^2 term
    hexq = ["-0x1.88e2ep-25", "0x1.036804p-23", "-0x1.a91a98p-25", "0x1.224e4cp-23", "0x1.3c8ae2p-23"]
    hexr = ["0x1.6d458p-1", "-0x1.149cd8p-2", "0x1.5196a2p-1", "-0x1.ee575ap-3", "-0x1.c55e2p-3"]
    q = np.array([[float.fromhex(v) for v in hexq]], dtype=f32)
    r = np.array([[float.fromhex(v) for v in hexr]], dtype=f32)
    h = 0.4502110246667935
    rn, ro = expanded_ratios(q, r, np.zeros((1, 5), f32), h)
    assert ro[0] > 1.0, ro[0]          # 9.26 / 9
    assert rn[0] <= 1.0, rn[0]


@pytest.mark.parametrize("D", [1, 3, 5])
def test_radius_criterion_per_term_error(D):
    # a run admitted by (10 D + 32) u rho_Q^2 / 2h^2 <= E has per-term error
    # at most E + (4 D + 8) u x, x = |q - r|^2 / 2h^2
    rng = np.random.default_rng(300 + D)
    n = 50000
    rho, h = 0.05, 0.1
    m = np.full((1, D), 0.5, f32)
    dirs = rng.standard_normal((n, D))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    q = (m + dirs * rho * rng.random((n, 1)) ** (1.0 / D)).astype(f32)
    r = (m + (rng.random((n, D)) - 0.5) * 2.0).astype(f32)
    xh, qt, _ = expanded_exponent(q, r, m, h)
    rho_q2 = float((qt.astype(f64) ** 2).sum(1).max())
    E = (10 * D + 32) * U * rho_q2 / (2 * h * h)
    x = ((q.astype(f64) - r.astype(f64)) ** 2).sum(1) / (2 * h * h)
    err = np.abs(xh + LOG2E * x) / LOG2E
    assert np.all(err <= (E + (4 * D + 8) * U * x) * (1.0 + 1e-3))
