"""The log-mean polynomials of the CUDA kernels, read from the header and
checked on the CPU against 40-digit values of the functions they replace.

The device code evaluates ln_mean(x, y) = (s/2) Q(f2) and 1/ln_mean(x, y) =
S(f2)/s with s = x + y, f2 = ((y - x)/s)^2, S(f2) = 2 atanh(t)/t =
2 sum_k f2^k/(2k+1) and Q = 2/S (the logarithmic mean of Ranocha's flux,
Sec. 3.2 of the paper; ln(y/x) = 2 atanh t). Here S is summed from its
series in decimal arithmetic, the header's coefficients are taken exactly as
the doubles they are, and the relative error over each polynomial's interval
must stay within the bound its comment states."""
import os
import re
import struct
from decimal import Decimal, getcontext

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2108_06476_gb300", "csrc")
HEADER = os.path.join(CSRC, "dg_device.cuh")
HEADER32 = os.path.join(CSRC, "dg_f32.cuh")
getcontext().prec = 40


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


def polynomial(text, real, name):
    """(coefficients lowest order first, interval end, stated error)."""
    sig = f"{real} {name}({real} f2)"
    body = _body(text, sig)
    comment = text[:text.rfind("\n", 0, text.index(sig))].splitlines()[-1]
    m = re.search(r"degree (\d+) on f2 in \[0, ([0-9.e-]+)\]; measured relative error ([0-9.e-]+)",
                  comment)
    assert m, comment
    lits = re.findall(r"(-?\d+\.\d*(?:e-?\d+)?)f?[;)]", body)
    coeffs = [float(x) for x in lits][::-1]
    if real == "float":
        assert all(float(np.float32(c)) == c for c in coeffs)
    assert len(coeffs) == int(m.group(1)) + 1
    return coeffs, Decimal(m.group(2)), float(m.group(3))


def S_ref(f2):
    total, term, k = Decimal(0), Decimal(1), 0
    while term > Decimal("1e-45") or k < 2:
        total += term / (2 * k + 1)
        term *= f2
        k += 1
    return 2 * total


def Q_ref(f2):
    return 2 / S_ref(f2)


def R_ref(f2):
    """R = (1 - Q)/f2, the polynomial of the FP32 perturbation form."""
    if f2 == 0:
        return Decimal(1) / 3
    return (1 - Q_ref(f2)) / f2


POLYS = [("double", "q_short", Q_ref, 2e-19), ("double", "s_short", S_ref, 5e-19),
         ("double", "q_long", Q_ref, 2e-17), ("double", "s_long", S_ref, 1e-17)]
# the FP32 kernels' perturbation form: FP64 small-difference branch and the
# FP32 range
# (the FP64 branch's first-order series stays 40x below the FP32 rounding)
POLYS32 = [("double", "phi_r64", R_ref, 1.5e-9), ("float", "phi_r32", R_ref, 5e-8)]


def _check_accuracy(text, real, name, ref, cap):
    coeffs, a, stated = polynomial(text, real, name)
    assert stated <= cap
    exact = [Decimal(c) for c in coeffs]
    worst = Decimal(0)
    n = 600
    for k in range(n + 1):
        x = a * k / n
        p = Decimal(0)
        for c in reversed(exact):
            p = p * x + c
        worst = max(worst, abs(p / ref(x) - 1))
    assert float(worst) <= 1.05 * stated, (name, float(worst))
    return coeffs


@pytest.mark.parametrize("real,name,ref,cap", POLYS, ids=[f"{p[0]}-{p[1]}" for p in POLYS])
def test_polynomial_accuracy(header, real, name, ref, cap):
    coeffs = _check_accuracy(header, real, name, ref, cap)
    assert coeffs[0] == (1.0 if name.startswith("q") else 2.0)  # ln_mean(x, x) = x exactly


@pytest.mark.parametrize("real,name,ref,cap", POLYS32, ids=[f"{p[0]}-{p[1]}" for p in POLYS32])
def test_perturbation_form_polynomials(real, name, ref, cap):
    with open(HEADER32) as fh:
        text = fh.read()
    coeffs = _check_accuracy(text, real, name, ref, cap)
    # the divided-difference evaluator uses the same coefficients
    fn = "void phi_r64_dd(double a" if real == "double" else "void phi_r32_dd(float a"
    body = _body(text, fn)
    lits = [float(x) for x in re.findall(r"(-?\d+\.\d*(?:e-?\d+)?)f?[;)]", body)]
    assert set(lits) == set(coeffs), (lits, coeffs)


def test_series_limit_of_the_fp64_branch():
    with open(HEADER32) as fh:
        text = fh.read()
    lim = float(re.search(r"kSeriesLim = ([0-9.e-]+)f;", text).group(1))
    assert lim == 1.0e-4  # the oracle's series threshold
    assert float(polynomial(text, "double", "phi_r64")[1]) >= lim


def test_series_reference_is_the_logarithmic_mean():
    # Q_ref(f2) with x = 1 - t, y = 1 + t (s/2 = 1) against (y - x)/ln(y/x)
    for t in ("0.01", "0.1", "0.3", "0.49"):
        t = Decimal(t)
        lm = 2 * t / ((1 + t) / (1 - t)).ln()
        assert abs(Q_ref(t * t) / lm - 1) < Decimal("1e-35")


def test_range_limits(header):
    for value, name in ((1e-2, "in_short"), (0.25, "in_long")):
        body = _body(header, f"bool {name}(double f2)")
        bits = int(re.search(r"0x([0-9A-F]+)LL", body).group(1), 16)
        assert struct.unpack("<q", struct.pack("<d", value))[0] == bits
    # every polynomial covers the range that selects it
    for name, lim in (("q_short", 1e-2), ("s_short", 1e-2), ("q_long", 0.25), ("s_long", 0.25)):
        assert float(polynomial(header, "double", name)[1]) >= lim


# The FP64 kernels evaluate the short-range polynomials with their tail in
# FP32 (q_short_mixed from f2^4, s_short_mixed from f2^5): the same
# coefficients, the tail's rounded to FP32, and the evaluation (f2 truncated
# to FP32, FP32 Horner tail, FP64 Horner head) within 3e-17 of Q and 2e-18
# of S over [0, 1e-2], emulated here with exact decimal arithmetic and FP32
# rounding of every tail operation.
def _f32(x):
    return Decimal(float(np.float32(float(x))))


def _f32_trunc(x):
    """x >= 0 truncated to FP32 (the kernels' conversion of f2)."""
    d = float(x)
    f = np.float32(d)
    if float(f) > d:
        f = np.nextafter(f, np.float32(0))
    return Decimal(float(f))


@pytest.mark.parametrize("name,mixed,split,ref,bound",
                         [("q_short", "q_short_mixed", 4, Q_ref, 3e-17),
                          ("s_short", "s_short_mixed", 5, S_ref, 2e-18)])
def test_mixed_precision_short_polynomials(header, name, mixed, split, ref, bound):
    coeffs = polynomial(header, "double", name)[0]
    body = _body(header, f"double {mixed}(double f2)")
    # the tail's literals carry the f suffix (rounded to FP32 by the
    # compiler) and are the double coefficients as written; the head's are
    # the double coefficients
    flits = [float(x) for x in re.findall(r"(-?\d+\.\d*(?:e-?\d+)?)f[;),]", body)]
    dlits = [float(x) for x in re.findall(r"(-?\d+\.\d*(?:e-?\d+)?)[;),]", body)]
    assert sorted(flits) == sorted(coeffs[split:]), (flits, coeffs)
    assert sorted(dlits) == sorted(coeffs[:split]), (dlits, coeffs)
    tail = [float(np.float32(c)) for c in coeffs[split:]]
    head = coeffs[:split]
    worst = Decimal(0)
    for k in range(401):
        x = Decimal(1e-2) * k / 400
        xf = _f32_trunc(x)
        t = Decimal(tail[-1])
        for c in reversed(tail[:-1]):
            t = _f32(xf * t + Decimal(c))  # one FP32 fused multiply-add
        p = t
        for c in reversed(head):
            p = p * x + Decimal(c)
        worst = max(worst, abs(p / ref(x) - 1))
    assert float(worst) <= bound, (mixed, float(worst))
