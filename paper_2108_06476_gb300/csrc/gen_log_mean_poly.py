"""Writes the polynomial coefficients of the log-mean kernels (C++ text on
stdout, pasted into dg_device.cuh).

The logarithmic mean of Ranocha's flux (Sec. 3.2 of the paper cites the
evaluation of ranocha2021efficient) is written with s = x + y,
t = (y - x)/s and f2 = t^2, using ln(y/x) = 2 atanh(t):
    ln_mean(x, y)   = (s/2) Q(f2),  Q(f2) = t / atanh(t),
    1/ln_mean(x, y) = S(f2) / s,    S(f2) = 2 atanh(t) / t.
Both are analytic in f2 on [0, 1). On an interval [0, a] each is replaced by
a polynomial c_0 + f2 r(f2) with c_0 = Q(0) = 1 or S(0) = 2 exactly (so that
ln_mean(x, x) = x), where r interpolates (F(f2) - c_0)/f2 at the Chebyshev
points of [0, a]: close to the best uniform approximation of that degree,
with far fewer terms than the Taylor series for the same error. The script
evaluates Q and S with 60-digit arithmetic (mpmath) and prints each
polynomial's degree, interval, coefficients (rounded to the kernel's type)
and the largest relative error it measured on a dense grid.

Usage: python gen_log_mean_poly.py
"""
import mpmath as mp
import numpy as np

mp.mp.dps = 60

# (name, function, real type, interval end, degree)
POLYS = [
    ("q_short", "Q", "double", "1e-2", 6),
    ("s_short", "S", "double", "1e-2", 6),
    ("q_long", "Q", "double", "0.25", 13),
    ("s_long", "S", "double", "0.25", 14),
]

# the FP32 kernels' perturbation form (dg_f32.cuh) uses R(f2) = (1 - Q(f2))/f2
# (phi = 1 - Q = f2 R): its FP32 range is a plain interpolant of R at the
# Chebyshev points of [0, 0.25], rounded to FP32; its FP64 small-difference
# branch (f2 < 1e-4) is the Taylor series of R to first order, printed by
# series_r(2) (its truncation, 1.4e-9 relative, lies far below the FP32
# rounding of the results it feeds).
R_POLYS = [("phi_r32", "float", "0.25", 5)]


def Q(f2):
    if f2 == 0:
        return mp.mpf(1)
    t = mp.sqrt(f2)
    return t / mp.atanh(t)


def S(f2):
    if f2 == 0:
        return mp.mpf(2)
    t = mp.sqrt(f2)
    return 2 * mp.atanh(t) / t


def R(f2):
    if f2 == 0:
        return mp.mpf(1) / 3
    return (1 - Q(f2)) / f2


def fit_plain(fun, a, degree):
    """Monomial coefficients interpolating fun at degree + 1 Chebyshev points."""
    nodes = [a * (1 + mp.cos(mp.pi * (2 * k + 1) / (2 * (degree + 1)))) / 2
             for k in range(degree + 1)]
    V = mp.matrix([[x ** j for j in range(degree + 1)] for x in nodes])
    c = mp.lu_solve(V, mp.matrix([fun(x) for x in nodes]))
    return [c[j] for j in range(degree + 1)]


def series_r(terms=4):
    """Taylor coefficients of R(f2): 1/Q = sum_k f2^k/(2k+1) inverted."""
    s = [mp.mpf(1) / (2 * k + 1) for k in range(terms + 2)]
    inv = [mp.mpf(1)]  # coefficients of Q = 1/s
    for n in range(1, terms + 2):
        inv.append(-sum(s[k] * inv[n - k] for k in range(1, n + 1)))
    return [-inv[k + 1] for k in range(terms)]  # R = (1 - Q)/f2


def fit(fun, a, degree):
    """Monomial coefficients c_0..c_degree (60 digits)."""
    c0 = fun(0)
    nodes = [a * (1 + mp.cos(mp.pi * (2 * k + 1) / (2 * degree))) / 2 for k in range(degree)]
    V = mp.matrix([[x ** j for j in range(degree)] for x in nodes])
    r = mp.lu_solve(V, mp.matrix([(fun(x) - c0) / x for x in nodes]))
    return [c0] + [r[j] for j in range(degree)]


def rounded(coeffs, real):
    if real == "double":
        return [float(c) for c in coeffs]
    return [float(np.float32(float(c))) for c in coeffs]


def max_rel_error(fun, coeffs, a, points=2000):
    worst = mp.mpf(0)
    for k in range(points + 1):
        x = a * k / points
        p = mp.mpf(0)
        for c in reversed(coeffs):
            p = p * x + mp.mpf(c)
        worst = max(worst, abs(p / fun(x) - 1))
    return float(worst)


def c_function(name, real, coeffs, a, err):
    suffix, fma = ("f", "fmaf") if real == "float" else ("", "fma")
    lit = [repr(c) + suffix for c in coeffs]
    lines = [f"// degree {len(coeffs) - 1} on f2 in [0, {a}]; measured relative error {err:.1e}",
             f"__device__ __forceinline__ {real} {name}({real} f2) {{",
             f"  {real} r = {lit[-1]};"]
    for c in reversed(lit[1:-1]):
        lines.append(f"  r = {fma}(f2, r, {c});")
    lines.append(f"  return {fma}(f2, r, {lit[0]});")
    lines.append("}")
    return "\n".join(lines)


def main():
    for name, fname, real, a, degree in POLYS:
        fun = {"Q": Q, "S": S}[fname]
        coeffs = rounded(fit(fun, mp.mpf(a), degree), real)
        print(c_function(name, real, coeffs, a, max_rel_error(fun, coeffs, mp.mpf(a))))
    for name, real, a, degree in R_POLYS:
        coeffs = rounded(fit_plain(R, mp.mpf(a), degree), real)
        print(c_function(name, real, coeffs, a, max_rel_error(R, coeffs, mp.mpf(a))))
    coeffs = [float(c) for c in series_r(2)]
    print(c_function("phi_r64", "double", coeffs, "1e-4",
                     max_rel_error(R, coeffs, mp.mpf("1e-4"))))


if __name__ == "__main__":
    main()
