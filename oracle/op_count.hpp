/*
 * Operation-counting scalar for the oracle's counting build (TEST
 * INFRASTRUCTURE ONLY, like the oracle itself): a double that adds one to a
 * global counter for every +, -, *, / it takes part in and for every log1p
 * and sqrt. Comparisons, negation and copies are not counted. Compiling
 * dgsem_oracle.c with real = counted (as C++, -DOR_COUNT) counts the
 * arithmetic of the oracle's formulas as written, which is the algorithmic
 * work per evaluation (a logarithm, a division or a square root as one
 * operation).
 */
#pragma once
#include <math.h>

extern long long or_op_count;

struct counted {
  double v;
  counted() : v(0.0) {}
  counted(double x) : v(x) {}
  counted& operator+=(const counted& o) { ++or_op_count; v += o.v; return *this; }
  counted& operator-=(const counted& o) { ++or_op_count; v -= o.v; return *this; }
  counted& operator*=(const counted& o) { ++or_op_count; v *= o.v; return *this; }
  counted& operator/=(const counted& o) { ++or_op_count; v /= o.v; return *this; }
};

inline counted operator+(const counted& a, const counted& b) { ++or_op_count; return counted(a.v + b.v); }
inline counted operator-(const counted& a, const counted& b) { ++or_op_count; return counted(a.v - b.v); }
inline counted operator*(const counted& a, const counted& b) { ++or_op_count; return counted(a.v * b.v); }
inline counted operator/(const counted& a, const counted& b) { ++or_op_count; return counted(a.v / b.v); }
inline counted operator+(const counted& a, double b) { return a + counted(b); }
inline counted operator-(const counted& a, double b) { return a - counted(b); }
inline counted operator*(const counted& a, double b) { return a * counted(b); }
inline counted operator/(const counted& a, double b) { return a / counted(b); }
inline counted operator+(double a, const counted& b) { return counted(a) + b; }
inline counted operator-(double a, const counted& b) { return counted(a) - b; }
inline counted operator*(double a, const counted& b) { return counted(a) * b; }
inline counted operator/(double a, const counted& b) { return counted(a) / b; }
inline counted operator-(const counted& a) { return counted(-a.v); }
inline bool operator==(const counted& a, const counted& b) { return a.v == b.v; }
inline bool operator<(const counted& a, const counted& b) { return a.v < b.v; }

inline counted counted_log1p(const counted& x) { ++or_op_count; return counted(log1p(x.v)); }
inline counted counted_sqrt(const counted& x) { ++or_op_count; return counted(sqrt(x.v)); }
