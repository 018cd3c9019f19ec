"""Pins for the oracle's Hermite functions (Section 3.1).

h_n(t) = e^{-t^2} H_n(t) is computed in the oracle by the three-term
recurrence.  It is pinned here by the polynomials the paper prints, by
Rodrigues' formula differentiated symbolically, by the generating-function
identity and by Szasz's inequality used in the truncation lemmas.
"""
import math

import numpy as np
import pytest
import sympy as sp

from conftest import read_golden

T_GRID = np.linspace(-4.0, 4.0, 33)


def test_paper_printed_polynomials(orc):
    # H_0 = 1, H_1 = 2t, H_2 = 4t^2 - 2 (Section 3.1).
    for row in read_golden("hermite_polynomials.txt"):
        n, coef = int(row[0]), row[1:]
        for t in T_GRID:
            Hn = sum(c * t ** k for k, c in enumerate(coef))
            got = orc.hermite_functions(t, n + 1)[n]
            assert got == pytest.approx(math.exp(-t * t) * Hn, rel=1e-13, abs=1e-300)


@pytest.mark.parametrize("n", range(0, 12))
def test_rodrigues_formula(orc, n):
    # H_n(t) = (-1)^n e^{t^2} d^n/dt^n e^{-t^2}, so h_n(t) = (-1)^n d^n/dt^n e^{-t^2}.
    t = sp.Symbol("t")
    deriv = sp.lambdify(t, (-1) ** n * sp.diff(sp.exp(-t ** 2), t, n), "math")
    for tv in T_GRID:
        want = float(deriv(float(tv)))
        got = orc.hermite_functions(float(tv), n + 1)[n]
        scale = max(1.0, abs(want))
        assert abs(got - want) <= 1e-11 * scale * (n + 1)


@pytest.mark.parametrize("s", [-0.9, -0.3, 0.0, 0.45, 1.0])
def test_generating_function(orc, s):
    # e^{-(t-s)^2} = sum_n s^n/n! h_n(t)  (the generating function times e^{-t^2}).
    for t in T_GRID:
        hn = orc.hermite_functions(t, 40)
        series = sum(s ** n / math.factorial(n) * hn[n] for n in range(40))
        assert series == pytest.approx(math.exp(-(t - s) ** 2), rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("h", [0.05, 0.7, 3.0])
def test_scaled_shifted_1d_expansion(orc, h):
    # e^{-(t-s)^2/2h^2} = sum_n (1/n!) ((s-s0)/sqrt(2h^2))^n h_n((t-s0)/sqrt(2h^2)).
    rng = np.random.default_rng(5)
    k = 1.0 / math.sqrt(2 * h * h)
    for _ in range(20):
        s0 = rng.uniform(-1, 1) * h
        s = s0 + rng.uniform(-0.8, 0.8) * h
        t = s0 + rng.uniform(-5, 5) * h
        hn = orc.hermite_functions((t - s0) * k, 40)
        series = sum(((s - s0) * k) ** n / math.factorial(n) * hn[n] for n in range(40))
        assert series == pytest.approx(math.exp(-(t - s) ** 2 / (2 * h * h)), rel=1e-10, abs=1e-14)


def test_szasz_inequality(orc):
    # |h_n(x)|/n! <= 2^{n/2}/sqrt(n!) e^{-x^2/2}, used by the truncation lemmas.
    for x in np.linspace(-6, 6, 121):
        hn = orc.hermite_functions(x, 16)
        for n in range(16):
            lhs = abs(hn[n]) / math.factorial(n)
            rhs = 2 ** (n / 2) / math.sqrt(math.factorial(n)) * math.exp(-x * x / 2)
            assert lhs <= rhs * (1 + 1e-12) + 1e-300
