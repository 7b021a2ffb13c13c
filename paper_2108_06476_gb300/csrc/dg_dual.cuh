// Forward-mode dual numbers for the flux Jacobians of the rhs
// vector-Jacobian product: a value and K partial derivatives, propagated
// through + - * / fma sqrt log1p and the reciprocal. Comparisons, max, min
// and |.| act on the value; max and min take the first argument on ties and
// d|x|/dx = sign(x) with sign(0) = +1 (the subgradient convention of the
// oracle's complex-step derivative).
#pragma once
#include "dg_device.cuh"

namespace dg {

template <typename R, int K>
struct Dual {
  R v;
  R d[K];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(R x) : v(x) {
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = R(0);
  }
};

#define DG_DUAL template <typename R, int K> __device__ __forceinline__

__device__ __forceinline__ double log1p_(double z) { return ::log1p(z); }
__device__ __forceinline__ float log1p_(float z) { return ::log1pf(z); }

DG_DUAL Dual<R, K> operator+(const Dual<R, K>& a, const Dual<R, K>& b) {
  Dual<R, K> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
DG_DUAL Dual<R, K> operator-(const Dual<R, K>& a, const Dual<R, K>& b) {
  Dual<R, K> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
DG_DUAL Dual<R, K> operator-(const Dual<R, K>& a) {
  Dual<R, K> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
  return r;
}
DG_DUAL Dual<R, K> operator*(const Dual<R, K>& a, const Dual<R, K>& b) {
  Dual<R, K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = ::fma(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
DG_DUAL Dual<R, K> operator/(const Dual<R, K>& a, const Dual<R, K>& b) {
  Dual<R, K> r;
  const R ib = R(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
// mixed with plain scalars
DG_DUAL Dual<R, K> operator+(const Dual<R, K>& a, R b) { Dual<R, K> r = a; r.v += b; return r; }
DG_DUAL Dual<R, K> operator+(R b, const Dual<R, K>& a) { Dual<R, K> r = a; r.v += b; return r; }
DG_DUAL Dual<R, K> operator-(const Dual<R, K>& a, R b) { Dual<R, K> r = a; r.v -= b; return r; }
DG_DUAL Dual<R, K> operator-(R b, const Dual<R, K>& a) { return Dual<R, K>(b) - a; }
DG_DUAL Dual<R, K> operator*(const Dual<R, K>& a, R b) {
  Dual<R, K> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b;
  return r;
}
DG_DUAL Dual<R, K> operator*(R b, const Dual<R, K>& a) { return a * b; }
DG_DUAL Dual<R, K> operator/(const Dual<R, K>& a, R b) { return a * (R(1) / b); }
DG_DUAL Dual<R, K> operator/(R a, const Dual<R, K>& b) { return Dual<R, K>(a) / b; }
DG_DUAL Dual<R, K>& operator+=(Dual<R, K>& a, const Dual<R, K>& b) { a = a + b; return a; }
DG_DUAL Dual<R, K>& operator-=(Dual<R, K>& a, const Dual<R, K>& b) { a = a - b; return a; }
DG_DUAL bool operator<(const Dual<R, K>& a, const Dual<R, K>& b) { return a.v < b.v; }
DG_DUAL bool operator<=(const Dual<R, K>& a, const Dual<R, K>& b) { return a.v <= b.v; }
DG_DUAL bool operator>=(const Dual<R, K>& a, const Dual<R, K>& b) { return a.v >= b.v; }
DG_DUAL bool operator>(const Dual<R, K>& a, const Dual<R, K>& b) { return a.v > b.v; }
DG_DUAL bool operator<(const Dual<R, K>& a, R b) { return a.v < b; }
DG_DUAL bool operator<=(const Dual<R, K>& a, R b) { return a.v <= b; }
DG_DUAL bool operator>=(const Dual<R, K>& a, R b) { return a.v >= b; }
DG_DUAL bool operator>(const Dual<R, K>& a, R b) { return a.v > b; }

DG_DUAL Dual<R, K> rn_mul(const Dual<R, K>& a, const Dual<R, K>& b) { return a * b; }
DG_DUAL Dual<R, K> rn_add(const Dual<R, K>& a, const Dual<R, K>& b) { return a + b; }
DG_DUAL Dual<R, K> rn_sub(const Dual<R, K>& a, const Dual<R, K>& b) { return a - b; }
DG_DUAL Dual<R, K> fma(const Dual<R, K>& a, const Dual<R, K>& b, const Dual<R, K>& c) {
  return a * b + c;
}
DG_DUAL Dual<R, K> fma(R a, const Dual<R, K>& b, const Dual<R, K>& c) { return a * b + c; }
DG_DUAL Dual<R, K> fma(const Dual<R, K>& a, const Dual<R, K>& b, R c) { return a * b + c; }
DG_DUAL Dual<R, K> fma(const Dual<R, K>& a, R b, R c) { return a * b + c; }
DG_DUAL Dual<R, K> fma(const Dual<R, K>& a, R b, const Dual<R, K>& c) { return a * b + c; }
DG_DUAL Dual<R, K> sqrt(const Dual<R, K>& a) {
  Dual<R, K> r;
  r.v = ::sqrt(a.v);
  const R h = R(0.5) / r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * h;
  return r;
}
DG_DUAL Dual<R, K> rcp(const Dual<R, K>& a) {
  Dual<R, K> r;
  r.v = R(1) / a.v;
  const R s = -r.v * r.v;
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * s;
  return r;
}
DG_DUAL Dual<R, K> log1p_(const Dual<R, K>& a) {
  Dual<R, K> r;
  r.v = log1p_(a.v);
  const R s = R(1) / (R(1) + a.v);
#pragma unroll
  for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * s;
  return r;
}
DG_DUAL Dual<R, K> fmax(const Dual<R, K>& a, const Dual<R, K>& b) { return a.v >= b.v ? a : b; }
DG_DUAL Dual<R, K> fmin(const Dual<R, K>& a, const Dual<R, K>& b) { return a.v <= b.v ? a : b; }
DG_DUAL Dual<R, K> fabs(const Dual<R, K>& a) { return a.v < R(0) ? -a : a; }

DG_DUAL Dual<R, K> series_q(const Dual<R, K>& f2) {
  // Taylor coefficients of t / atanh t in powers of f2 through f2^7
  // (truncation below 2e-18 for f2 < 1e-2; log1p beyond)
  const R c[8] = {R(1.0), R(-1.0 / 3.0), R(-4.0 / 45.0), R(-44.0 / 945.0), R(-428.0 / 14175.0),
                  R(-10196.0 / 467775.0), R(-10719068.0 / 638512875.0),
                  R(-25865068.0 / 1915538625.0)};
  Dual<R, K> q(c[7]);
#pragma unroll
  for (int i = 6; i >= 0; --i) q = q * f2 + c[i];
  return q;
}
DG_DUAL Dual<R, K> series_s(const Dual<R, K>& f2) {
  Dual<R, K> s(R(2.0 / 15.0));
  const R c[7] = {R(2.0), R(2.0 / 3.0), R(2.0 / 5.0), R(2.0 / 7.0), R(2.0 / 9.0), R(2.0 / 11.0),
                  R(2.0 / 13.0)};
#pragma unroll
  for (int i = 6; i >= 0; --i) s = s * f2 + c[i];
  return s;
}
DG_DUAL R series_limit(const Dual<R, K>&) { return series_limit(R(0)); }

DG_DUAL Dual<R, K> ln_mean(const Dual<R, K>& x, const Dual<R, K>& y) {
  const Dual<R, K> s = x + y;
  const Dual<R, K> t = (y - x) * rcp(s);
  const Dual<R, K> f2 = t * t;
  if (f2.v < series_limit(R(0))) return R(0.5) * s * series_q(f2);
  return (y - x) / log1p_((y - x) / x);
}
DG_DUAL Dual<R, K> inv_ln_mean(const Dual<R, K>& x, const Dual<R, K>& y) {
  const Dual<R, K> rs = rcp(x + y);
  const Dual<R, K> t = (y - x) * rs;
  const Dual<R, K> f2 = t * t;
  if (f2.v < series_limit(R(0))) return series_s(f2) * rs;
  return log1p_((y - x) / x) / (y - x);
}

#undef DG_DUAL

}  // namespace dg
