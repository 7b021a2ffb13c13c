// Device-side building blocks of the DGSEM rhs: mesh/basis parameters, the
// conserved-to-primitive prologue, the logarithmic mean, the two-point volume
// fluxes and the surface fluxes, all templated on the arithmetic type R
// (double or float). Kernels live in dg_rhs_kernels.cuh.
//
// Formulas (paper: Ranocha et al., "Adaptive numerical simulations with
// Trixi.jl", Sec. 2.1 and 3.1, which cite them):
//   Euler flux     f_n(u) = (rho v_n, rho v_n v + p e_n, (E + p) v_n),
//                  p = (gamma - 1)(E - rho |v|^2 / 2)
//   log mean       ln_mean(x, y) = (y - x) / ln(y / x) (ranocha2021efficient's
//                  atanh-series idea, with a longer series and log1p)
//   Ranocha EC/KEP flux (ranocha2020icosahom), Chandrashekar EC flux,
//   central flux (weak form, gassner2016split), local Lax-Friedrichs and HLL.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dg {

constexpr int kNPMax = 8;  // N <= 7
// Cartesian FP64 meshes with fewer elements than this (about four per SM)
// run the pair-parallel volume kernel, and a whole rhs or stage as one launch
constexpr long long kPairParallelElems = 4 * 152;

// error-word bits
constexpr unsigned kErrRho = 1u, kErrP = 2u, kErrNaN = 4u;

struct Geom {
  int n[3];         // elements per direction (1 for unused)
  long long nelem;  // total elements (< 2^31)
  double gamma;
  double gm1;       // gamma - 1
  double gm1inv;    // 1 / (gamma - 1)
};

// Per-direction split-form tables, scaled by the inverse Jacobian:
//   Ds[k][a][b] = -(2/h_k) Dt[a][b], Dt = 2 D - W^-1 B (zero diagonal)
//   liftR[k] = -(2/h_k)/w_N (right face), liftL[k] = +(2/h_k)/w_0 (left face)
template <typename R>
struct Tables {
  R Ds[3][kNPMax][kNPMax];
  R liftR[3];
  R liftL[3];
};

// The split-form and lifting coefficients of the dimension's directions,
// times sc, into a shared copy (every thread of the block calls it; a
// barrier must follow before use). A fused stage passes sc = dt, so that the
// line sums are dt du itself and the epilogue needs no product by dt; the
// rhs alone passes 1, which leaves every coefficient exact.
template <int D, int N, typename R>
__device__ __forceinline__ void stage_tables(Tables<R>& dst, const Tables<R>& tb, R sc) {
  constexpr int NP = N + 1;
  for (int t = threadIdx.x; t < D * NP * NP; t += blockDim.x) {
    const int dir = t / (NP * NP), a = (t / NP) % NP, b = t % NP;
    dst.Ds[dir][a][b] = sc * tb.Ds[dir][a][b];
  }
  if ((int)threadIdx.x < D) {
    dst.liftR[threadIdx.x] = sc * tb.liftR[threadIdx.x];
    dst.liftL[threadIdx.x] = sc * tb.liftL[threadIdx.x];
  }
}

// Optional fusion of the Runge-Kutta stage into the volume kernel's
// epilogue: with k set, du is not stored; instead k <- a k + dt du and
// u <- u + b k for the element (the surface kernel of the same stage has
// already read every trace, and no other CTA reads this element's u).
// ref (FP32 meshes only): the per-element FP32 reference states of the
// perturbation form (dg_f32.cuh), (d+2) floats per element, written by the
// reference kernel before the surface kernel and read by both flux kernels.
struct StageFuse {
  double* k = nullptr;
  const double* dt = nullptr;
  double a = 0.0, b = 0.0;
  float* ref = nullptr;
  double* refE = nullptr;   // FP32 meshes: the references' FP64 energies
  double* u_out = nullptr;  // where u + b k goes (nullptr: u, in place)
};

template <int D, int N>
struct Shape {
  static constexpr int NP = N + 1;
  static constexpr int P = (D == 2) ? NP * NP : NP * NP * NP;  // nodes per element
  static constexpr int NV = D + 2;                              // conserved variables
  static constexpr int LINES = P / NP;                          // lines per direction
};

// Node index of position a along direction DIR on line l (l enumerates the
// remaining coordinates in ascending order, first one fastest). The same l
// enumerates the face nodes of the two faces normal to DIR.
template <int D, int N, int DIR>
__device__ __forceinline__ int line_node(int l, int a) {
  constexpr int NP = N + 1;
  if (DIR == 0) return a + NP * l;
  if (DIR == 1) return (D == 2) ? l + NP * a : (l % NP) + NP * a + NP * NP * (l / NP);
  return l + NP * NP * a;
}

template <int D, int N>
__device__ __forceinline__ int line_node_rt(int dir, int l, int a) {
  if (dir == 0) return line_node<D, N, 0>(l, a);
  if (dir == 1) return line_node<D, N, 1>(l, a);
  return line_node<D, N, 2>(l, a);
}

// Neighbour of element e at offset +-1 in direction dir (periodic).
__device__ __forceinline__ long long neighbour(const Geom& g, long long e, int dir, int s) {
  long long ex = e % g.n[0];
  long long r = e / g.n[0];
  long long ey = r % g.n[1];
  long long ez = r / g.n[1];
  if (dir == 0) ex = (ex + s + g.n[0]) % g.n[0];
  else if (dir == 1) ey = (ey + s + g.n[1]) % g.n[1];
  else ez = (ez + s + g.n[2]) % g.n[2];
  return ex + (long long)g.n[0] * (ey + (long long)g.n[1] * ez);
}

// ---- rounding-explicit scalar ops (used where both sides of a comparison
// or a cancellation must round identically to a plain IEEE evaluation) ----
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }

// ---- reciprocals ----
// FP64: hardware approximation (rcp.approx.ftz.f64, about 2^-22 relative)
// refined by one third-order Newton step r <- r (1 + e + e^2), e = 1 - x r,
// which cubes the relative error; within about one ulp of 1/x for normal x.
__device__ __forceinline__ double rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}
// FP32: the hardware approximation (rcp.approx.ftz.f32, within 1 ulp).
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <typename R, int D>
struct Prim {
  R rho, v[D], p;
};

// Primitive variables from conserved ones, rounded as the plain left-to-right
// IEEE evaluation of v_k = m_k / rho, p = (gamma-1) (E - (rho/2) |v|^2).
// The quotients use one reciprocal and a residual correction
// q = m r + (m - rho (m r)) r, which gives the correctly rounded m / rho.
template <typename R, int D>
__device__ __forceinline__ Prim<R, D> cons2prim(const R* c, R gm1) {
  Prim<R, D> q;
  q.rho = c[0];
  const R rr = rcp(c[0]);
  R v2 = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const R q0 = c[1 + k] * rr;
    q.v[k] = fma(fma(-c[0], q0, c[1 + k]), rr, q0);
    v2 = (k == 0) ? rn_mul(q.v[0], q.v[0]) : rn_add(v2, rn_mul(q.v[k], q.v[k]));
  }
  q.p = rn_mul(gm1, rn_sub(c[D + 1], rn_mul(rn_mul(R(0.5), c[0]), v2)));
  return q;
}

// Primitive variables for the flux and time-step kernels: one reciprocal
// rr = 1/rho (kept for the sound speed), v_k = m_k rr and
// p = (gamma-1) (E - m.v/2) with fused products. The fluxes' rounding is
// dominated by the pressure terms and the time step needs a few ulp, so the
// quotients need no correction there.
template <int D>
__device__ __forceinline__ Prim<double, D> prim_rcp(const double* c, double gm1, double& rr) {
  Prim<double, D> q;
  q.rho = c[0];
  rr = rcp(c[0]);
  double mv = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    q.v[k] = c[1 + k] * rr;
    mv = fma(c[1 + k], q.v[k], mv);
  }
  q.p = gm1 * fma(-0.5, mv, c[D + 1]);
  return q;
}

template <typename R, int D>
__device__ __forceinline__ unsigned prim_check(const Prim<R, D>& q) {
  unsigned bad = 0;
  if (!(q.rho > R(0))) bad |= kErrRho;
  if (!(q.p > R(0))) bad |= kErrP;
  if (!isfinite(q.rho) || !isfinite(q.p)) bad |= kErrNaN;
  return bad;
}
// the same tests of doubles on their bit patterns (integer pipe): x > 0
// for 0 < bits <= bits of +inf, finite unless the exponent field is all ones
template <int D>
__device__ __forceinline__ unsigned prim_check(const Prim<double, D>& q) {
  constexpr long long kInf = 0x7ff0000000000000LL;
  const long long r = __double_as_longlong(q.rho), p = __double_as_longlong(q.p);
  unsigned bad = 0;
  if (!(r > 0 && r <= kInf)) bad |= kErrRho;
  if (!(p > 0 && p <= kInf)) bad |= kErrP;
  if ((r & kInf) == kInf || (p & kInf) == kInf) bad |= kErrNaN;
  return bad;
}

// ---- FP64 <-> FP32 conversions on the integer pipe ----
// The FP64 pipe (2 lanes per clock per SM on this part) also executes the
// hardware conversions between double and float, which would otherwise take
// a third of the FP64 work of the FP32 kernels (and the FP64 kernels'
// polynomial tails below). These rebuild the IEEE 754
// bit patterns instead (binary64: 1 sign, 11 exponent bits with bias 1023,
// 52 fraction bits; binary32: 1, 8 with bias 127, 23): for results in the
// normal range and for zeros; everything else (subnormals, overflow, inf,
// NaN) takes the hardware conversion out of line.
static __device__ __noinline__ float d2f_slow(double x) { return (float)x; }
static __device__ __noinline__ double f2d_slow(float x) { return (double)x; }

// double -> float, rounded to nearest (ties to even)
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 253u) {  // float exponent 1..253: no overflow after rounding
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 fraction bits
    const unsigned rest = lo & 0x1fffffffu;                   // the 29 dropped bits
    unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | m;
    f += (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));  // carries into e
    return __uint_as_float(f);
  }
  if (((hi << 1) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);  // +-0
  return d2f_slow(x);
}

// float -> double (exact)
__device__ __forceinline__ double f2d(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned fe = (b >> 23) & 0xffu;
  if (fe - 1u < 254u)  // normal
    return __hiloint2double((int)((b & 0x80000000u) | ((fe + 896u) << 20) | ((b & 0x7fffffu) >> 3)),
                            (int)(b << 29));
  if ((b << 1) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);  // +-0
  return f2d_slow(x);
}

// ---- halving ----
// x / 2 of a double by decrementing its exponent field on the integer pipe:
// exact, the same value as 0.5 * x, for normal x above the smallest
// exponent; infinities, NaNs and zeros are their own halves; subnormal and
// smallest-exponent values (never met in practice) take the multiplication
// out of line. The FP64 kernels are bound by their FP64 unit.
static __device__ __noinline__ double half_slow(double x) { return 0.5 * x; }
__device__ __forceinline__ double half(double x) {
  const long long b = __double_as_longlong(x);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if (e - 2u < 0x7fdu) return __longlong_as_double(b - (1LL << 52));
  if (e == 0x7ffu || (b << 1) == 0) return x;
  return half_slow(x);
}
__device__ __forceinline__ float half(float x) { return 0.5f * x; }

// max of two non-negative doubles (magnitudes, squared speeds) by their bit
// patterns on the integer pipe: the order of non-negative IEEE values is
// that of their bits, and a NaN (sign bit clear) exceeds every number, so it
// is the result (fmax would drop it)
__device__ __forceinline__ double fmax_nn(double a, double b) {
  return __double_as_longlong(a) >= __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ float fmax_nn(float a, float b) { return fmaxf(a, b); }

// ---- square root of a positive double (wave speeds) ----
// Goldschmidt's coupled iteration for g = sqrt(x) and h = 1/(2 sqrt(x)), in
// the form given by P. Markstein, "Software division and square root using
// Goldschmidt's algorithms" (2004), from the hardware reciprocal square root
// approximation y (rsqrt.approx.ftz.f64): g = x y, h = y/2; one step
// r = 1/2 - g h, g += g r, h += h r squares the relative error, and the
// correction g += (x - g^2) h squares it again, leaving the rounding of the
// last FMA: within one ulp of the correctly rounded root, with six FP64
// instructions. Positive normal arguments only; zero, negative, subnormal,
// infinite and NaN arguments take the library square root out of line.
static __device__ __noinline__ double sqrt_slow(double x) { return sqrt(x); }
__device__ __forceinline__ double sqrt_pos(double x) {
  const long long b = __double_as_longlong(x);
  // positive normal: bits in [2^52, 0x7ff0000000000000)
  if ((unsigned long long)(b - (1LL << 52)) >= 0x7fe0000000000000ULL) return sqrt_slow(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double g = x * y, h = half(y);
  const double r = fma(-g, h, 0.5);
  g = fma(g, r, g);
  h = fma(h, r, h);
  return fma(fma(-g, g, x), h, g);
}
__device__ __forceinline__ float sqrt_pos(float x) { return sqrtf(x); }

// ---- logarithmic mean ----
// ln_mean(x, y) = (y - x) / ln(y / x). With s = x + y, t = (y - x)/s and
// f2 = t^2, ln(y/x) = 2 atanh(t), so
//   ln_mean(x, y)   = (s/2) Q(f2),   Q(f2) = t / atanh(t),
//   1/ln_mean(x, y) = S(f2) / s,     S(f2) = 2 atanh(t) / t = 2 sum_k f2^k/(2k+1).
// For f2 < 1/9 (y/x in [1/2, 2]) y - x is exact (Sterbenz); beyond, its
// rounding reaches Q and S only through f2, damped by 2 f2 |dQ/df2| < 0.2.
// Every rounding is relative to the result; in the far range
// ln(y/x) = log1p((y - x)/x). No form divides a rounding error by ln(y/x),
// which the flux differencing would amplify by (2/h)|Dt||f|/|du|, and the
// polynomial forms divide nothing.
//
// Three ranges of f2, each lane choosing its own (no result depends on the
// other lanes of its warp):
//   short  a low-degree polynomial (f2 < 1e-2),
//   long   a higher-degree one on [0, 0.25],
//   far    log1p.
// (These are the FP64 kernels' log means; the FP32 kernels use the
// perturbation form of dg_f32.cuh.)
// Each polynomial is c_0 + f2 r(f2) with c_0 = Q(0) = 1 or S(0) = 2 exactly
// and r interpolating (F - c_0)/f2 at the Chebyshev points of its interval
// (gen_log_mean_poly.py writes them): degree 6 where the Taylor series
// needs 7 for 1e-19 on [0, 1e-2], and degree 13-14 for 1e-17 on [0, 0.25],
// where it needs about 25. The stated errors are
// relative, of the coefficients as rounded, against 60-digit values.
// degree 6 on f2 in [0, 1e-2]; measured relative error 1.9e-19
__device__ __forceinline__ double q_short(double f2) {
  double r = -0.01719901874634888;
  r = fma(f2, r, -0.021792151641765893);
  r = fma(f2, r, -0.030194027707754922);
  r = fma(f2, r, -0.0465608465041037);
  r = fma(f2, r, -0.08888888888893755);
  r = fma(f2, r, -0.3333333333333333);
  return fma(f2, r, 1.0);
}
// degree 6 on f2 in [0, 1e-2]; measured relative error 4.5e-19
__device__ __forceinline__ double s_short(double f2) {
  double r = 0.15791323599162152;
  r = fma(f2, r, 0.18177218144198024);
  r = fma(f2, r, 0.22222246134174709);
  r = fma(f2, r, 0.28571428515311326);
  r = fma(f2, r, 0.4000000000004813);
  r = fma(f2, r, 0.6666666666666666);
  return fma(f2, r, 2.0);
}
// q_short and s_short with the terms of high degree summed in FP32, the
// rest by the same Horner scheme in FP64 (the FP64 kernels are bound by
// their FP64 unit; the FP32 pipe has room): Q from f2^4 (|c_4| f2^4 <=
// 3e-10 on [0, 1e-2], so the tail's FP32 rounding, with f2 truncated to
// FP32, stays below 3e-17 of Q),
// S from f2^5 (below 2e-18 of S). Same coefficients, the tail's rounded to
// FP32.
// f2 >= 0 as a float, its bit pattern truncated (0 below the float range):
// branch-free integer work, relative error below 2^-23 (the tail bound
// above allows for it)
__device__ __forceinline__ float f32_trunc_nonneg(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = hi >> 20;  // sign bit clear
  const unsigned f = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return e - 897u < 253u ? __uint_as_float(f) : 0.0f;
}
// a normal float as a double (exact; the tails are never zero or subnormal)
__device__ __forceinline__ double f64_of_normal(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned fe = (b >> 23) & 0xffu;
  return __hiloint2double((int)((b & 0x80000000u) | ((fe + 896u) << 20) | ((b & 0x7fffffu) >> 3)),
                          (int)(b << 29));
}
__device__ __forceinline__ double q_short_mixed(double f2) {
  const float f = f32_trunc_nonneg(f2);
  float t = -0.01719901874634888f;
  t = fmaf(f, t, -0.021792151641765893f);
  t = fmaf(f, t, -0.030194027707754922f);
  double r = fma(f2, f64_of_normal(t), -0.0465608465041037);
  r = fma(f2, r, -0.08888888888893755);
  r = fma(f2, r, -0.3333333333333333);
  return fma(f2, r, 1.0);
}
__device__ __forceinline__ double s_short_mixed(double f2) {
  const float f = f32_trunc_nonneg(f2);
  const float t = fmaf(f, 0.15791323599162152f, 0.18177218144198024f);
  double r = fma(f2, f64_of_normal(t), 0.22222246134174709);
  r = fma(f2, r, 0.28571428515311326);
  r = fma(f2, r, 0.4000000000004813);
  r = fma(f2, r, 0.6666666666666666);
  return fma(f2, r, 2.0);
}
// degree 13 on f2 in [0, 0.25]; measured relative error 1.1e-17
__device__ __forceinline__ double q_long(double f2) {
  double r = -0.02924278002496948;
  r = fma(f2, r, 0.015352807394837298);
  r = fma(f2, r, -0.017544611482937886);
  r = fma(f2, r, -0.005229417291853292);
  r = fma(f2, r, -0.010090678154396803);
  r = fma(f2, r, -0.011129369170977035);
  r = fma(f2, r, -0.013509289236067104);
  r = fma(f2, r, -0.016787171057780347);
  r = fma(f2, r, -0.02179681821069115);
  r = fma(f2, r, -0.030194003213882256);
  r = fma(f2, r, -0.04656084656443126);
  r = fma(f2, r, -0.08888888888887284);
  r = fma(f2, r, -0.33333333333333337);
  return fma(f2, r, 1.0);
}
// degree 14 on f2 in [0, 0.25]; measured relative error 4.8e-18
__device__ __forceinline__ double s_long(double f2) {
  double r = 0.42196195771951595;
  r = fma(f2, r, -0.28900982366828937);
  r = fma(f2, r, 0.27115807827384597);
  r = fma(f2, r, 0.024584897457081062);
  r = fma(f2, r, 0.10883830836469174);
  r = fma(f2, r, 0.10321539762294324);
  r = fma(f2, r, 0.11786199385180084);
  r = fma(f2, r, 0.1333177270540377);
  r = fma(f2, r, 0.15384691880541276);
  r = fma(f2, r, 0.18181815763018377);
  r = fma(f2, r, 0.22222222267877936);
  r = fma(f2, r, 0.2857142857098021);
  r = fma(f2, r, 0.4000000000000173);
  r = fma(f2, r, 0.6666666666666666);
  return fma(f2, r, 2.0);
}

__device__ __forceinline__ double series_limit(double) { return 1.0e-2; }
__device__ __forceinline__ float series_limit(float) { return 4.0e-2f; }

// far from x = y: the direct forms (rare; kept out of line)
static __device__ __noinline__ double ln_mean_far(double x, double y) { return (y - x) / log1p((y - x) / x); }
static __device__ __noinline__ float ln_mean_far(float x, float y) { return (y - x) / log1pf((y - x) / x); }
static __device__ __noinline__ double inv_ln_mean_far(double x, double y) { return log1p((y - x) / x) / (y - x); }
static __device__ __noinline__ float inv_ln_mean_far(float x, float y) { return log1pf((y - x) / x) / (y - x); }

// f2 >= 0 (an FP64 value in both kernel precisions), so the range tests
// compare IEEE bit patterns on the integer pipe (the FP64 pipe is the
// bottleneck of the FP64 kernels)
__device__ __forceinline__ bool in_short(double f2) {
  return __double_as_longlong(f2) < 0x3F847AE147AE147BLL;  // bits of 1e-2
}
__device__ __forceinline__ bool in_long(double f2) {
  return __double_as_longlong(f2) < 0x3FD0000000000000LL;  // bits of 0.25
}

// f2 = t^2 in FP64 for a t of either precision, and the Q and S of its range
// (second argument: the kernel precision)
__device__ __forceinline__ double f2_of(double t) { return t * t; }
__device__ __forceinline__ double f2_of(float t) {
  const double td = t;
  return td * td;
}
// MIXED: the short range's tails in FP32 (the default, which every kernel
// takes); false gives the FP64 polynomials of the same ranges
template <bool MIXED = true>
__device__ __forceinline__ double q_of(double f2, double) {
  double q;
  if (in_short(f2))
    q = MIXED ? q_short_mixed(f2) : q_short(f2);
  else
    q = q_long(f2);
  return q;
}
template <bool MIXED = true>
__device__ __forceinline__ double s_of(double f2, double) {
  double S;
  if (in_short(f2))
    S = MIXED ? s_short_mixed(f2) : s_short(f2);
  else
    S = s_long(f2);
  return S;
}
template <typename R>
__device__ __forceinline__ R ln_mean(R x, R y) {
  const R s = x + y;
  const R t = (y - x) * rcp(s);
  const double f2 = f2_of(t);
  if (!in_long(f2)) return ln_mean_far(x, y);
  return R(0.5) * s * q_of<>(f2, R(0));
}

template <typename R>
__device__ __forceinline__ R inv_ln_mean(R x, R y) {
  const R rs = rcp(x + y);
  const R t = (y - x) * rs;
  const double f2 = f2_of(t);
  if (!in_long(f2)) return inv_ln_mean_far(x, y);
  return s_of<>(f2, R(0)) * rs;
}

// ln_mean(2 hx, 2 hy) from the halves: every step is the one of
// ln_mean(x, y) scaled by an exact factor 2, so the result is bitwise
// ln_mean(x, y), without the product (x + y)/2.
template <typename R, bool MIXED = true>
__device__ __forceinline__ R ln_mean_halves(R hx, R hy) {
  const R hs = hx + hy;
  const R t = (hy - hx) * rcp(hs);
  const double f2 = f2_of(t);
  if (!in_long(f2)) return R(2) * ln_mean_far(hx, hy);
  return hs * q_of<MIXED>(f2, R(0));
}

// a + 1/ln_mean(x, y), the last product fused into the addition
template <typename R, bool MIXED = true>
__device__ __forceinline__ R add_inv_ln_mean(R x, R y, R a) {
  const R rs = rcp(x + y);
  const R t = (y - x) * rs;
  const double f2 = f2_of(t);
  if (!in_long(f2)) return a + inv_ln_mean_far(x, y);
  return fma(s_of<MIXED>(f2, R(0)), rs, a);
}

// ---- two-point volume fluxes f#(L, R) in direction DIR ----
enum { kVRanocha = 0, kVChandrashekar = 1, kVCentral = 2 };

template <typename R, int D, int DIR>
__device__ __forceinline__ void flux_ranocha(const Prim<R, D>& L, const Prim<R, D>& Rt, R gm1inv,
                                             R f[D + 2]) {
  const R rho_mean = ln_mean(L.rho, Rt.rho);
  const R inv_rho_p_mean = L.p * Rt.p * inv_ln_mean(L.rho * Rt.p, Rt.rho * L.p);
  R v_dot = L.v[0] * Rt.v[0];
#pragma unroll
  for (int k = 1; k < D; ++k) v_dot += L.v[k] * Rt.v[k];
  const R p_avg = R(0.5) * (L.p + Rt.p);
  f[0] = rho_mean * R(0.5) * (L.v[DIR] + Rt.v[DIR]);
#pragma unroll
  for (int k = 0; k < D; ++k) f[1 + k] = f[0] * R(0.5) * (L.v[k] + Rt.v[k]);
  f[1 + DIR] += p_avg;
  f[D + 1] = f[0] * (R(0.5) * v_dot + inv_rho_p_mean * gm1inv) +
             R(0.5) * (L.p * Rt.v[DIR] + Rt.p * L.v[DIR]);
}

template <typename R, int D, int DIR>
__device__ __forceinline__ void flux_chandrashekar(const Prim<R, D>& L, const Prim<R, D>& Rt,
                                                   R gm1inv, R f[D + 2]) {
  const R bL = R(0.5) * L.rho / L.p, bR = R(0.5) * Rt.rho / Rt.p;
  const R rho_ln = ln_mean(L.rho, Rt.rho), inv_beta_ln = inv_ln_mean(bL, bR);
  const R rho_avg = R(0.5) * (L.rho + Rt.rho), beta_avg = R(0.5) * (bL + bR);
  R v2L = R(0), v2R = R(0), va[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v2L += L.v[k] * L.v[k];
    v2R += Rt.v[k] * Rt.v[k];
    va[k] = R(0.5) * (L.v[k] + Rt.v[k]);
  }
  const R p_mean = R(0.5) * rho_avg / beta_avg;
  f[0] = rho_ln * va[DIR];
#pragma unroll
  for (int k = 0; k < D; ++k) f[1 + k] = f[0] * va[k];
  f[1 + DIR] += p_mean;
  R fe = f[0] * R(0.5) * (gm1inv * inv_beta_ln - R(0.5) * (v2L + v2R));
#pragma unroll
  for (int k = 0; k < D; ++k) fe += f[1 + k] * va[k];
  f[D + 1] = fe;
}

// physical flux from primitives (volume kernels keep only primitives)
template <typename R, int D, int DIR>
__device__ __forceinline__ void euler_flux_prim(const Prim<R, D>& q, R gm1inv, R f[D + 2]) {
  const R m = q.rho * q.v[DIR];
  R v2 = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) v2 += q.v[k] * q.v[k];
  f[0] = m;
#pragma unroll
  for (int k = 0; k < D; ++k) f[1 + k] = m * q.v[k];
  f[1 + DIR] += q.p;
  const R E = q.p * gm1inv + R(0.5) * q.rho * v2;
  f[D + 1] = (E + q.p) * q.v[DIR];
}

template <typename R, int D, int DIR>
__device__ __forceinline__ void flux_central(const Prim<R, D>& L, const Prim<R, D>& Rt, R gm1inv,
                                             R f[D + 2]) {
  R fl[D + 2], fr[D + 2];
  euler_flux_prim<R, D, DIR>(L, gm1inv, fl);
  euler_flux_prim<R, D, DIR>(Rt, gm1inv, fr);
#pragma unroll
  for (int v = 0; v < D + 2; ++v) f[v] = R(0.5) * (fl[v] + fr[v]);
}

template <int VF, typename R, int D, int DIR>
__device__ __forceinline__ void volume_flux(const Prim<R, D>& L, const Prim<R, D>& Rt, R gm1inv,
                                            R f[D + 2]) {
  if (VF == kVRanocha) flux_ranocha<R, D, DIR>(L, Rt, gm1inv, f);
  else if (VF == kVChandrashekar) flux_chandrashekar<R, D, DIR>(L, Rt, gm1inv, f);
  else flux_central<R, D, DIR>(L, Rt, gm1inv, f);
}

// ---- surface fluxes F*(u_L, u_R) in direction dir (runtime) ----
enum { kSLLF = 0, kSRanocha = 1, kSHLL = 2, kSChandrashekar = 3 };

// physical flux from the conserved state and its primitives
template <typename R, int D>
__device__ __forceinline__ void euler_flux_cons(const R* c, const Prim<R, D>& q, int dir,
                                                R f[D + 2]) {
  const R m = c[1 + dir];
  f[0] = m;
#pragma unroll
  for (int k = 0; k < D; ++k) f[1 + k] = m * q.v[k];
  f[1 + dir] += q.p;
  f[D + 1] = (c[D + 1] + q.p) * q.v[dir];
}

template <typename R, int D, int DIR>
__device__ __forceinline__ void surface_flux_dir(int sf, const R* cL, const R* cR,
                                                 const Prim<R, D>& L, const Prim<R, D>& Rt,
                                                 R gamma, R gm1inv, R f[D + 2]) {
  if (sf == kSRanocha) {
    flux_ranocha<R, D, DIR>(L, Rt, gm1inv, f);
    return;
  }
  if (sf == kSChandrashekar) {
    flux_chandrashekar<R, D, DIR>(L, Rt, gm1inv, f);
    return;
  }
  R fl[D + 2], fr[D + 2];
  euler_flux_cons<R, D>(cL, L, DIR, fl);
  euler_flux_cons<R, D>(cR, Rt, DIR, fr);
  const R cl = sqrt(gamma * L.p / L.rho), cr = sqrt(gamma * Rt.p / Rt.rho);
  if (sf == kSLLF) {
    const R lam = fmax(fabs(L.v[DIR]), fabs(Rt.v[DIR])) + fmax(cl, cr);
#pragma unroll
    for (int v = 0; v < D + 2; ++v) f[v] = R(0.5) * (fl[v] + fr[v]) - R(0.5) * lam * (cR[v] - cL[v]);
    return;
  }
  // HLL
  const R sL = fmin(L.v[DIR] - cl, Rt.v[DIR] - cr);
  const R sR = fmax(L.v[DIR] + cl, Rt.v[DIR] + cr);
#pragma unroll
  for (int v = 0; v < D + 2; ++v) {
    if (sL >= R(0)) f[v] = fl[v];
    else if (sR <= R(0)) f[v] = fr[v];
    else f[v] = (sR * fl[v] - sL * fr[v] + sL * sR * (cR[v] - cL[v])) / (sR - sL);
  }
}

}  // namespace dg
