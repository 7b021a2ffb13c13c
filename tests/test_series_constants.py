"""The log-mean series constants of the CUDA kernels, read from the header
and checked on the CPU against exact rational arithmetic.

The device code evaluates ln_mean(x, y) = (s/2) Q(f2) and 1/ln_mean(x, y) =
S(f2)/s, with s = x + y, f2 = ((y - x)/s)^2, S(f2) = 2 atanh(t)/t =
2 sum_k f2^k/(2k+1) and Q = 1/(S/2) (the logarithmic mean of Ranocha's flux,
Sec. 2 of the paper; the series follows from ln(y/x) = 2 atanh t). Q's
coefficients are rebuilt here by inverting the power series of atanh(t)/t
with fractions; the range limits are checked against their bit patterns and
the truncation bounds the header states."""
import math
import os
import re
import struct
from fractions import Fraction

import numpy as np
import pytest

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "paper_2108_06476_gb300", "csrc", "dg_device.cuh")

K = 24
A = [Fraction(1, 2 * k + 1) for k in range(K)]  # atanh(t)/t in powers of f2
Q = [Fraction(1)] + [Fraction(0)] * (K - 1)
for _n in range(1, K):
    Q[_n] = -sum(A[j] * Q[_n - j] for j in range(1, _n + 1))
S = [2 * a for a in A]


@pytest.fixture(scope="module")
def header():
    with open(HEADER) as fh:
        return fh.read()


def _body(text, signature):
    i = text.index(signature)
    j = text.index("{", i)
    depth, k = 0, j
    while True:
        depth += {"{": 1, "}": -1}.get(text[k], 0)
        if depth == 0:
            return text[j:k + 1]
        k += 1


def _value(expr):
    expr = re.sub(r"(\d)f\b", r"\1", expr.strip())
    assert re.fullmatch(r"[-+0-9.e/ ]+", expr), expr
    return eval(expr)  # a literal or a quotient of two literals


def coefficients(text, signature):
    """Horner constants of one device function, lowest order first."""
    body = _body(text, signature)
    consts = []
    m = re.search(r"(?:double|float) \w+ = ([^;]+);", body)
    if m and "fma" not in m.group(1):
        consts.append(_value(m.group(1)))
    for m in re.finditer(r"fmaf?\(f2, \w+, ([^;]+?)\)(?:;|$)", body, re.M):
        consts.append(_value(m.group(1)))
    return consts[::-1]


CASES = [
    # (real, series, tail, exact coefficients, short terms, long terms, limits, rtol)
    ("double", "series_q", "series_q_tail", Q, 8, 20, (1e-2, 0.16), 2e-16),
    ("double", "series_s", "series_s_tail", S, 8, 21, (1e-2, 0.16), 2e-16),
    ("float", "series_q", "series_q_tail", Q, 6, 11, (4e-2, 0.25), 1e-7),
    ("float", "series_s", "series_s_tail", S, 6, 12, (4e-2, 0.25), 1e-7),
]


@pytest.mark.parametrize("real,series,tail,exact,n_short,n_long,limits,rtol", CASES)
def test_coefficients_are_the_series(header, real, series, tail, exact, n_short, n_long,
                                     limits, rtol):
    low = coefficients(header, f"{real} {series}({real} f2, {real} tail)")
    high = coefficients(header, f"{real} {tail}({real} f2)")
    assert len(low) == n_short and len(low) + len(high) == n_long
    for k, c in enumerate(low + high):
        assert abs(c - float(exact[k])) <= rtol * abs(float(exact[k])), (series, k)


@pytest.mark.parametrize("real,series,tail,exact,n_short,n_long,limits,rtol", CASES)
def test_truncation_within_stated_bounds(real, series, tail, exact, n_short, n_long, limits,
                                         rtol):
    # the coefficients' magnitudes never grow and every omitted term has
    # the sign of the first one, so the omitted sum is below
    # |first term| / (1 - f2) relative to the value at f2 = 0
    assert all(abs(exact[k + 1]) <= abs(exact[k]) for k in range(K - 1))
    bound = {"double": (6e-18, 6e-19), "float": (1e-9, 4e-9)}[real]
    for n, lim, b in ((n_short, limits[0], bound[0]), (n_long, limits[1], bound[1])):
        first = abs(exact[n]) * Fraction(lim) ** n
        assert float(first / (1 - Fraction(lim)) / abs(exact[0])) < b


def test_range_limits_bit_patterns(header):
    for value, name in ((1e-2, "in_short"), (0.16, "in_long")):
        body = _body(header, f"bool {name}(double f2)")
        bits = int(re.search(r"0x([0-9A-F]+)LL", body).group(1), 16)
        assert struct.unpack("<q", struct.pack("<d", value))[0] == bits
    assert "f2 < 4.0e-2f" in _body(header, "bool in_short(float f2)")
    assert "f2 < 0.25f" in _body(header, "bool in_long(float f2)")


def _horner(f2, coeffs):
    r = 0.0
    for c in reversed(coeffs):
        r = r * f2 + c
    return r


def test_long_range_log_mean_accuracy(header):
    """The long-range FP64 evaluation (tail, then the low-order part) matches
    the logarithmic mean to a few ulp over f2 in [1e-2, 0.16], and the short
    one over [0, 1e-2]; x = 1 - t and y = 1 + t make s = 2 and the reference
    2t / (log1p(t) - log1p(-t)), correct to about one ulp."""
    q_lo = coefficients(header, "double series_q(double f2, double tail)")
    q_hi = coefficients(header, "double series_q_tail(double f2)")
    s_lo = coefficients(header, "double series_s(double f2, double tail)")
    s_hi = coefficients(header, "double series_s_tail(double f2)")
    worst = 0.0
    for t in np.concatenate([np.linspace(0.0, 0.0999, 40), np.linspace(0.1, 0.3999, 60)]):
        f2 = t * t
        longer = f2 >= 1e-2
        qv = _horner(f2, q_lo + q_hi if longer else q_lo)
        sv = _horner(f2, s_lo + s_hi if longer else s_lo)
        # x = 1 - t, y = 1 + t: s = 2, ln_mean = 2 t / ln((1+t)/(1-t))
        exact = 1.0 if t == 0 else 2 * t / (math.log1p(t) - math.log1p(-t))
        worst = max(worst, abs(qv - exact) / exact, abs(sv / 2 - 1 / exact) * exact)
    assert worst < 2e-15
