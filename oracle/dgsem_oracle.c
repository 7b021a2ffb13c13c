/*
 * Plain, slow FP64 CPU oracle of the DGSEM right-hand side for the 2D/3D
 * compressible Euler equations on a uniform periodic Cartesian mesh, plus the
 * Carpenter-Kennedy low-storage RK stage, the CFL time step and the analysis
 * integrals.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it. It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * What it follows (paper: "Adaptive numerical simulations with Trixi.jl"):
 *   - the conservation law d_t u + sum_j d_xj f^j(u) = 0, Sec. 2, Eq. (1)
 *     (eq:hcl), with the ideal-gas compressible Euler equations named there;
 *   - the DGSEM of the cited texts (Kopriva 2009, Hesthaven-Warburton 2007),
 *     Sec. 2.1, on LGL nodes with collocated quadrature;
 *   - entropy-conservative split-form flux differencing (Sec. 2.1; Sec. 3.1,
 *     "flux differencing solver") with the EC/KEP flux of Ranocha
 *     (ranocha2020icosahom, ranocha2018thesis) and the logarithmic mean of
 *     ranocha2021efficient (Sec. 3.2);
 *   - local Lax-Friedrichs surface flux (Sec. 2.2 example, flux_lax_friedrichs)
 *     and HLL (Sec. 3.1, weak-form runs);
 *   - the 5-stage 4th-order low-storage RK of Carpenter and Kennedy and the
 *     CFL time step (Sec. 3.1);
 *   - the integrated quantities of the analysis callbacks (Sec. 2.2).
 * The paper writes none of these formulas out; each is restated here from
 * the published method it cites. Readings of open points are listed in the
 * repository's design notes.
 *
 * Structure: the rhs is the split form of the DGSEM (Fisher-Carpenter;
 * Gassner-Winters-Kopriva), per node and per coordinate direction,
 *     du_i = -(2/h) [ sum_m 2 D_im f#(u_i, u_m)
 *                     + (delta_iN (F*_R - f(u_i)) - delta_i0 (F*_L - f(u_i))) / w_i ],
 * evaluated in the algebraically identical form
 *     du_i = -(2/h) [ sum_m Dt_im f#(u_i, u_m) + delta_iN F*_R / w_N - delta_i0 F*_L / w_0 ]
 * with Dt = 2 D - W^-1 B formed in long double (see or_dtilde): the first
 * form cancels 2 D_00 f(u_0) against f(u_0)/w_0 in floating point at every
 * boundary node. Every two-point flux is evaluated for the node it updates
 * (both orders of each pair, and m = i), every surface flux once per adjacent
 * element. No pair halving, no blocking, no reordering.
 *
 * The file is compiled twice: once with real = double (names or_*), once with
 * real = double complex and -DOR_CSTEP (names orc_*), which gives the exact
 * Jacobian-vector product of the rhs by complex-step differentiation
 * (or_rhs_jvp). Comparisons and the non-smooth max/abs act on real parts.
 * Build with -ffp-contract=off so that no fused multiply-add changes rounding.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef OR_CSTEP
#include <complex.h>
typedef double complex real;
#define OR(name) orc_##name
#define RE(x) creal(x)
#define RLOG1P(x) clog(1.0 + (x))
#define RSQRT(x) csqrt(x)
#elif defined(OR_LONGDOUBLE)
/* extended-precision build (names orl_*): the same operator evaluated in long
 * double, used by the tests to measure the FP64 evaluations' rounding errors */
typedef long double real;
#define OR(name) orl_##name
#define RE(x) (x)
#define RLOG1P(x) log1pl(x)
#define RSQRT(x) sqrtl(x)
#elif defined(OR_COUNT)
/* operation-counting build (names orn_*, compiled as C++): every +, -, *, /,
 * log1p and sqrt of real values adds one to or_op_count (op_count.hpp); the
 * orn_ops_* entry points below report the counts of the method's pieces */
#include "op_count.hpp"
typedef counted real;
#define OR(name) orn_##name
#define RE(x) ((x).v)
#define RLOG1P(x) counted_log1p(x)
#define RSQRT(x) counted_sqrt(x)
#else
typedef double real;
#define OR(name) or_##name
#define RE(x) (x)
#define RLOG1P(x) log1p(x)
#define RSQRT(x) sqrt(x)
#endif

/* |x| and max(a, b) decided on real parts (derivative: sign(x) with sign(0)=+1,
 * and the left argument on ties). */
static real r_abs(real x) { return RE(x) < 0.0 ? -x : x; }
static real r_max(real a, real b) { return RE(a) >= RE(b) ? a : b; }
static real r_min(real a, real b) { return RE(a) <= RE(b) ? a : b; }

#define MAXV 5 /* at most d + 2 = 5 conserved variables */

/* ------------------------------------------------------------------------ */
/* Basis: LGL nodes and weights, differentiation matrix (the double build     */
/* exports them; the long double build keeps its own static copy).           */
/* ------------------------------------------------------------------------ */
#if !defined(OR_CSTEP)
/* Legendre P_N(x) and P_N'(x) by the three-term recurrence, long double. */
static void legendre(int N, long double x, long double *p, long double *dp) {
  long double p0 = 1.0L, p1 = x, d0 = 0.0L, d1 = 1.0L;
  if (N == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int k = 2; k <= N; ++k) {
    long double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    long double d2 = d0 + (2 * k - 1) * p1; /* P'_k = P'_{k-2} + (2k-1) P_{k-1} */
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

/* Legendre-Gauss-Lobatto nodes xi_0 = -1 < ... < xi_N = 1 (the interior ones
 * are the roots of P_N') and weights w_i = 2 / (N (N+1) P_N(xi_i)^2), in long
 * double. Newton iteration on P_N' from Chebyshev-Gauss-Lobatto guesses;
 * P_N'' from Legendre's equation (1-x^2) P'' = 2x P' - N(N+1) P. */
static int lgl_ld(int N, long double *xi, long double *w) {
  if (N < 1 || N > 32) return -1;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int j = 0; j <= N; ++j) {
    long double x;
    if (j == 0) x = -1.0L;
    else if (j == N) x = 1.0L;
    else {
      x = -cosl(pi * j / N);
      for (int it = 0; it < 100; ++it) {
        long double p, dp;
        legendre(N, x, &p, &dp);
        long double d2p = (2.0L * x * dp - (long double)N * (N + 1) * p) / (1.0L - x * x);
        long double dx = dp / d2p;
        x -= dx;
        if (fabsl(dx) < 1e-30L) break;
      }
    }
    long double p, dp;
    legendre(N, x, &p, &dp);
    xi[j] = x;
    w[j] = 2.0L / ((long double)N * (N + 1) * p * p);
  }
  return 0;
}

#ifndef OR_LONGDOUBLE
int or_lgl(int N, double *xi, double *w) {
  long double x[33], ww[33];
  if (lgl_ld(N, x, ww)) return -1;
  for (int j = 0; j <= N; ++j) { xi[j] = (double)x[j]; w[j] = (double)ww[j]; }
  return 0;
}

#endif

/* Nodal differentiation matrix D_ij = l_j'(xi_i) (row-major, long double) from
 * barycentric weights; D_ii = -sum_{j != i} D_ij. */
static int dmat_ld(int N, const long double *xi, long double *D) {
  int np = N + 1;
  long double lam[64];
  if (np > 64) return -1;
  for (int j = 0; j < np; ++j) {
    long double prod = 1.0L;
    for (int k = 0; k < np; ++k)
      if (k != j) prod *= (xi[j] - xi[k]);
    lam[j] = 1.0L / prod;
  }
  for (int i = 0; i < np; ++i) {
    long double diag = 0.0L;
    for (int j = 0; j < np; ++j) {
      if (j == i) continue;
      long double v = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      D[i * np + j] = v;
      diag -= v;
    }
    D[i * np + i] = diag;
  }
  return 0;
}

#ifndef OR_LONGDOUBLE
/* D as doubles, from the double nodes xi (used by the basis pins). */
int or_diff_matrix(int N, const double *xi, double *D) {
  long double x[64], Dl[64 * 64];
  if (N < 1 || N > 63) return -1;
  for (int j = 0; j <= N; ++j) x[j] = xi[j];
  dmat_ld(N, x, Dl);
  for (int t = 0; t < (N + 1) * (N + 1); ++t) D[t] = (double)Dl[t];
  return 0;
}

/* Split-form volume matrix Dt = 2 D - W^-1 B with B = diag(-1, 0, ..., 0, 1),
 * formed in long double from the long double basis and rounded once. By the
 * summation-by-parts property W D + (W D)^T = B its diagonal vanishes, and
 *   sum_m 2 D_im f#(u_i,u_m) - (B_ii / w_i) f(u_i) = sum_m Dt_im f#(u_i,u_m)
 * since f#(u,u) = f(u); also returns the weights. */
int or_dtilde(int N, double *Dt, double *w) {
  long double x[33], ww[33], Dl[33 * 33];
  if (lgl_ld(N, x, ww)) return -1;
  dmat_ld(N, x, Dl);
  int np = N + 1;
  for (int i = 0; i < np; ++i) {
    for (int j = 0; j < np; ++j) {
      long double v = 2.0L * Dl[i * np + j];
      if (i == j && i == 0) v += 1.0L / ww[0];
      if (i == j && i == N) v -= 1.0L / ww[N];
      Dt[i * np + j] = (double)v;
    }
    w[i] = (double)ww[i];
  }
  return 0;
}

#endif

/* Split-form tables in the working precision: Dt = 2 D - W^-1 B and w. */
static int tables_real(int N, real *Dt, real *w) {
#ifdef OR_LONGDOUBLE
  long double x[33], ww[33], Dl[33 * 33];
  if (lgl_ld(N, x, ww)) return -1;
  dmat_ld(N, x, Dl);
  int np = N + 1;
  for (int i = 0; i < np; ++i) {
    for (int j = 0; j < np; ++j) {
      long double v = 2.0L * Dl[i * np + j];
      if (i == j && i == 0) v += 1.0L / ww[0];
      if (i == j && i == N) v -= 1.0L / ww[N];
      Dt[i * np + j] = v;
    }
    w[i] = ww[i];
  }
  return 0;
#else
  double Dd[256], wd[16];
  if (or_dtilde(N, Dd, wd)) return -1;
  for (int t = 0; t < (N + 1) * (N + 1); ++t) Dt[t] = Dd[t];
  for (int i = 0; i <= N; ++i) w[i] = wd[i];
  return 0;
#endif
}

#ifndef OR_LONGDOUBLE
/* Carpenter-Kennedy (1994) five-stage fourth-order 2N-storage RK, "solution 3":
 * k <- A_s k + dt rhs(u); u <- u + B_s k. c_s are the stage times. */
void or_lsrk_coefficients(double *A, double *B, double *c) {
  A[0] = 0.0;
  A[1] = -567301805773.0 / 1357537059087.0;
  A[2] = -2404267990393.0 / 2016746695238.0;
  A[3] = -3550918686646.0 / 2091501179385.0;
  A[4] = -1275806237668.0 / 842570457699.0;
  B[0] = 1432997174477.0 / 9575080441755.0;
  B[1] = 5161836677717.0 / 13612068292357.0;
  B[2] = 1720146321549.0 / 2090206949498.0;
  B[3] = 3134564353537.0 / 4481467310338.0;
  B[4] = 2277821191437.0 / 14882151754819.0;
  c[0] = 0.0;
  c[1] = 1432997174477.0 / 9575080441755.0;
  c[2] = 2526269341429.0 / 6820363962896.0;
  c[3] = 2006345519317.0 / 3224310063776.0;
  c[4] = 2802321613138.0 / 2924317926251.0;
}
#endif
#else
int or_lgl(int N, double *xi, double *w);
int or_dtilde(int N, double *Dt, double *w);
static int tables_real(int N, real *Dt, real *w) {
  double Dd[256], wd[16];
  if (or_dtilde(N, Dd, wd)) return -1;
  for (int t = 0; t < (N + 1) * (N + 1); ++t) Dt[t] = Dd[t];
  for (int i = 0; i <= N; ++i) w[i] = wd[i];
  return 0;
}
#endif

/* ------------------------------------------------------------------------ */
/* Compressible Euler, ideal gas: u = (rho, rho v_1..rho v_d, E).            */
/* ------------------------------------------------------------------------ */

/* Primitive state (rho, v_1..v_d, p), p = (gamma-1)(E - rho |v|^2 / 2). */
static void cons2prim(int d, double gamma_d, const real *u, real *rho, real *v, real *p) {
  const real gamma = gamma_d;
  *rho = u[0];
  real v2 = 0.0;
  for (int k = 0; k < d; ++k) {
    v[k] = u[1 + k] / u[0];
    v2 += v[k] * v[k];
  }
  *p = (gamma - 1.0) * (u[d + 1] - 0.5 * u[0] * v2);
}

/* Physical flux in direction n: (rho v_n, rho v_n v + p e_n, (E + p) v_n). */
void OR(euler_flux)(int d, int n, double gamma, const real *u, real *f) {
  real rho, v[3], p;
  cons2prim(d, gamma, u, &rho, v, &p);
  f[0] = u[1 + n];
  for (int k = 0; k < d; ++k) f[1 + k] = u[1 + n] * v[k];
  f[1 + n] += p;
  f[d + 1] = (u[d + 1] + p) * v[n];
}

/* Logarithmic mean (y - x) / ln(y / x) in the form of ranocha2021efficient:
 * with f2 = ((x - y) / (x + y))^2, a truncated series of the identity
 * ln(y/x) = 2 atanh((y - x)/(y + x)) for f2 < 1e-4, the direct quotient
 * otherwise. In the direct quotient ln(y/x) is evaluated as log1p((y-x)/x):
 * log(fl(y/x)) would carry the rounding of y/x divided by ln(y/x), up to
 * ~50 ulps just above the switch. */
real OR(ln_mean)(real x, real y) {
#ifdef OR_LONGDOUBLE
  /* extended precision: the direct form everywhere (no series truncation) */
  if (x == y) return x;
  return (y - x) / RLOG1P((y - x) / x);
#endif
  real f2 = (x * (x - 2.0 * y) + y * y) / (x * (x + 2.0 * y) + y * y);
  if (RE(f2) < 1.0e-4)
    return (x + y) / (2.0 + f2 * (2.0 / 3.0 + f2 * (2.0 / 5.0 + f2 * (2.0 / 7.0))));
  return (y - x) / RLOG1P((y - x) / x);
}

/* Ranocha's entropy-conserving and kinetic-energy-preserving two-point flux,
 * direction n (ranocha2020icosahom; used in volume and surface in Sec. 3.1):
 *   f_rho = ln_mean(rho) * avg(v_n)
 *   f_mk  = f_rho avg(v_k) + avg(p) delta_kn
 *   f_E   = f_rho (0.5 v_L.v_R + 1/((gamma-1) ln_mean(rho/p)))
 *           + 0.5 (p_L v_R,n + p_R v_L,n)
 * with 1/ln_mean(rho/p) = p_L p_R / ln_mean(rho_L p_R, rho_R p_L). */
void OR(flux_ranocha)(int d, int n, double gamma, const real *uL, const real *uR, real *f) {
  real rL, vL[3], pL, rR, vR[3], pR;
  cons2prim(d, gamma, uL, &rL, vL, &pL);
  cons2prim(d, gamma, uR, &rR, vR, &pR);
  real rho_mean = OR(ln_mean)(rL, rR);
  real inv_rho_p_mean = pL * pR / OR(ln_mean)(rL * pR, rR * pL);
  real v_dot = 0.0;
  for (int k = 0; k < d; ++k) v_dot += vL[k] * vR[k];
  real p_avg = 0.5 * (pL + pR);
  f[0] = rho_mean * 0.5 * (vL[n] + vR[n]);
  for (int k = 0; k < d; ++k) f[1 + k] = f[0] * 0.5 * (vL[k] + vR[k]);
  f[1 + n] += p_avg;
  f[d + 1] = f[0] * (0.5 * v_dot + inv_rho_p_mean / (gamma - 1.0)) +
             0.5 * (pL * vR[n] + pR * vL[n]);
}

/* Chandrashekar's entropy-conserving, kinetic-energy-preserving flux with
 * beta = rho / (2 p):
 *   f_rho = ln_mean(rho) avg(v_n)
 *   f_mk  = f_rho avg(v_k) + delta_kn avg(rho) / (2 avg(beta))
 *   f_E   = f_rho (1/(2 (gamma-1) ln_mean(beta)) - 0.5 avg(|v|^2)) + sum_k f_mk avg(v_k) */
void OR(flux_chandrashekar)(int d, int n, double gamma, const real *uL, const real *uR, real *f) {
  real rL, vL[3], pL, rR, vR[3], pR;
  cons2prim(d, gamma, uL, &rL, vL, &pL);
  cons2prim(d, gamma, uR, &rR, vR, &pR);
  real bL = 0.5 * rL / pL, bR = 0.5 * rR / pR;
  real rho_ln = OR(ln_mean)(rL, rR), beta_ln = OR(ln_mean)(bL, bR);
  real rho_avg = 0.5 * (rL + rR), beta_avg = 0.5 * (bL + bR);
  real v2L = 0.0, v2R = 0.0, va[3];
  for (int k = 0; k < d; ++k) {
    v2L += vL[k] * vL[k];
    v2R += vR[k] * vR[k];
    va[k] = 0.5 * (vL[k] + vR[k]);
  }
  real p_mean = 0.5 * rho_avg / beta_avg;
  f[0] = rho_ln * va[n];
  for (int k = 0; k < d; ++k) f[1 + k] = f[0] * va[k];
  f[1 + n] += p_mean;
  real fe = f[0] * 0.5 * (1.0 / ((gamma - 1.0) * beta_ln) - 0.5 * (v2L + v2R));
  for (int k = 0; k < d; ++k) fe += f[1 + k] * va[k];
  f[d + 1] = fe;
}

/* Central flux 0.5 (f(u_L) + f(u_R)); as a volume flux it gives the standard
 * weak-form DGSEM (Sec. 3.1, gassner2016split). */
void OR(flux_central)(int d, int n, double gamma, const real *uL, const real *uR, real *f) {
  real fL[MAXV], fR[MAXV];
  OR(euler_flux)(d, n, gamma, uL, fL);
  OR(euler_flux)(d, n, gamma, uR, fR);
  for (int v = 0; v < d + 2; ++v) f[v] = 0.5 * (fL[v] + fR[v]);
}

/* Local Lax-Friedrichs: 0.5 (f_L + f_R) - 0.5 lambda (u_R - u_L) with
 * lambda = max(|v_n,L|, |v_n,R|) + max(c_L, c_R), c = sqrt(gamma p / rho). */
void OR(flux_llf)(int d, int n, double gamma, const real *uL, const real *uR, real *f) {
  real rL, vL[3], pL, rR, vR[3], pR, fL[MAXV], fR[MAXV];
  cons2prim(d, gamma, uL, &rL, vL, &pL);
  cons2prim(d, gamma, uR, &rR, vR, &pR);
  OR(euler_flux)(d, n, gamma, uL, fL);
  OR(euler_flux)(d, n, gamma, uR, fR);
  real cL = RSQRT(gamma * pL / rL), cR = RSQRT(gamma * pR / rR);
  real lam = r_max(r_abs(vL[n]), r_abs(vR[n])) + r_max(cL, cR);
  for (int v = 0; v < d + 2; ++v) f[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

/* HLL with the signal-speed estimates S_L = min(v_n,L - c_L, v_n,R - c_R),
 * S_R = max(v_n,L + c_L, v_n,R + c_R):
 *   f_L if S_L >= 0, f_R if S_R <= 0, else
 *   (S_R f_L - S_L f_R + S_L S_R (u_R - u_L)) / (S_R - S_L). */
void OR(flux_hll)(int d, int n, double gamma, const real *uL, const real *uR, real *f) {
  real rL, vL[3], pL, rR, vR[3], pR, fL[MAXV], fR[MAXV];
  cons2prim(d, gamma, uL, &rL, vL, &pL);
  cons2prim(d, gamma, uR, &rR, vR, &pR);
  OR(euler_flux)(d, n, gamma, uL, fL);
  OR(euler_flux)(d, n, gamma, uR, fR);
  real cL = RSQRT(gamma * pL / rL), cR = RSQRT(gamma * pR / rR);
  real sL = r_min(vL[n] - cL, vR[n] - cR), sR = r_max(vL[n] + cL, vR[n] + cR);
  for (int v = 0; v < d + 2; ++v) {
    if (RE(sL) >= 0.0) f[v] = fL[v];
    else if (RE(sR) <= 0.0) f[v] = fR[v];
    else f[v] = (sR * fL[v] - sL * fR[v] + sL * sR * (uR[v] - uL[v])) / (sR - sL);
  }
}

typedef void (*two_point_flux)(int, int, double, const real *, const real *, real *);

/* Volume flux ids: 0 Ranocha, 1 Chandrashekar, 2 central (weak form). */
static two_point_flux volume_flux_by_id(int id) {
  switch (id) {
    case 0: return OR(flux_ranocha);
    case 1: return OR(flux_chandrashekar);
    case 2: return OR(flux_central);
    default: return 0;
  }
}
/* Surface flux ids: 0 LLF, 1 Ranocha (EC), 2 HLL, 3 Chandrashekar (EC). */
static two_point_flux surface_flux_by_id(int id) {
  switch (id) {
    case 0: return OR(flux_llf);
    case 1: return OR(flux_ranocha);
    case 2: return OR(flux_hll);
    case 3: return OR(flux_chandrashekar);
    default: return 0;
  }
}

/* Exported single-flux evaluators for the pins: kind 0..2 volume ids,
 * 10 + s for surface id s, 20 for the physical flux f(u_L). */
int OR(two_point)(int kind, int d, int n, double gamma, const real *uL, const real *uR, real *f) {
  two_point_flux fn = 0;
  if (kind >= 0 && kind < 10) fn = volume_flux_by_id(kind);
  else if (kind >= 10 && kind < 20) fn = surface_flux_by_id(kind - 10);
  else if (kind == 20) { OR(euler_flux)(d, n, gamma, uL, f); return 0; }
  if (!fn) return -1;
  fn(d, n, gamma, uL, uR, f);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Mesh indexing: uniform periodic Cartesian grid of n_0 x n_1 (x n_2)       */
/* elements on [lo_0,hi_0] x ...; element e = ex + n_0 (ey + n_1 ez); state */
/* u[e][v][k][j][i] with node i (x) fastest.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int d, N, np, nv;
  int n[3];
  long long nelem, P; /* elements, nodes per element */
  double h[3];
} mesh_t;

static int mesh_init(mesh_t *m, int d, int N, const int *n, const double *dom) {
  if (d < 2 || d > 3 || N < 1 || N > 15) return -1;
  m->d = d; m->N = N; m->np = N + 1; m->nv = d + 2;
  m->nelem = 1; m->P = 1;
  for (int k = 0; k < 3; ++k) { m->n[k] = 1; m->h[k] = 1.0; }
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1 || !(dom[2 * k + 1] > dom[2 * k])) return -1;
    m->n[k] = n[k];
    m->h[k] = (dom[2 * k + 1] - dom[2 * k]) / n[k];
    m->nelem *= n[k];
    m->P *= m->np;
  }
  return 0;
}

/* Element index of the neighbour of e at offset s = +-1 in direction dir. */
static long long neighbour(const mesh_t *m, long long e, int dir, int s) {
  int c[3];
  long long r = e;
  for (int k = 0; k < 3; ++k) { c[k] = (int)(r % m->n[k]); r /= m->n[k]; }
  c[dir] = (c[dir] + s + m->n[dir]) % m->n[dir];
  return c[0] + (long long)m->n[0] * (c[1] + (long long)m->n[1] * c[2]);
}

/* Node index with the coordinate in direction dir replaced by a. */
static long long node_with(const mesh_t *m, long long node, int dir, int a) {
  int c[3] = {0, 0, 0};
  long long r = node;
  for (int k = 0; k < m->d; ++k) { c[k] = (int)(r % m->np); r /= m->np; }
  c[dir] = a;
  long long out = 0;
  for (int k = m->d - 1; k >= 0; --k) out = out * m->np + c[k];
  return out;
}

static int node_coord(const mesh_t *m, long long node, int dir) {
  long long r = node;
  for (int k = 0; k < dir; ++k) r /= m->np;
  return (int)(r % m->np);
}

static void load_node(const mesh_t *m, const real *u, long long e, long long node, real *out) {
  for (int v = 0; v < m->nv; ++v) out[v] = u[(e * m->nv + v) * m->P + node];
}

/* ------------------------------------------------------------------------ */
/* The semidiscrete operator.                                               */
/* ------------------------------------------------------------------------ */

/* Directions whose volume and surface terms the rhs evaluates (bit k set:
 * direction k; all by default). du is the sum over directions of these
 * parts, so the parts of a state add up to its rhs; the tests use them to
 * measure how much an rhs cancels between directions. */
static int OR(dir_mask) = 7;
void OR(set_direction_mask)(int mask) { OR(dir_mask) = mask; }

/* du = rhs(u) for the elements listed in elems (all elements when elems is
 * NULL); du is written only for those elements. Returns 0, or -1 on bad
 * arguments. Split-form DGSEM, see the file header. */
int OR(rhs)(int d, int N, const int *n, const double *dom, double gamma, int vflux, int sflux,
            const real *u, real *du, const long long *elems, long long n_elems, int nthreads) {
  mesh_t m;
  if (mesh_init(&m, d, N, n, dom)) return -1;
  two_point_flux fvol = volume_flux_by_id(vflux), fsurf = surface_flux_by_id(sflux);
  if (!fvol || !fsurf) return -1;
  real w[16], Dt[256];
  tables_real(N, Dt, w);
  long long count = elems ? n_elems : m.nelem;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (long long t = 0; t < count; ++t) {
    long long e = elems ? elems[t] : t;
    for (long long node = 0; node < m.P; ++node) {
      real ui[MAXV], acc[MAXV];
      load_node(&m, u, e, node, ui);
      for (int v = 0; v < m.nv; ++v) acc[v] = 0.0;
      for (int dir = 0; dir < d; ++dir) {
        if (!((OR(dir_mask) >> dir) & 1)) continue;
        int i = node_coord(&m, node, dir);
        real vol[MAXV], f[MAXV], um[MAXV];
        for (int v = 0; v < m.nv; ++v) vol[v] = 0.0;
        /* volume: sum_m Dt_im f#(u_i, u_m) along the line */
        for (int a = 0; a <= N; ++a) {
          load_node(&m, u, e, node_with(&m, node, dir, a), um);
          fvol(d, dir, gamma, ui, um, f);
          for (int v = 0; v < m.nv; ++v) vol[v] += Dt[i * m.np + a] * f[v];
        }
        /* surface: + F*_R / w_N at the right face, - F*_L / w_0 at the left */
        if (i == N) {
          real fs[MAXV], uo[MAXV];
          load_node(&m, u, neighbour(&m, e, dir, +1), node_with(&m, node, dir, 0), uo);
          fsurf(d, dir, gamma, ui, uo, fs);
          for (int v = 0; v < m.nv; ++v) vol[v] += fs[v] / w[N];
        }
        if (i == 0) {
          real fs[MAXV], uo[MAXV];
          load_node(&m, u, neighbour(&m, e, dir, -1), node_with(&m, node, dir, N), uo);
          fsurf(d, dir, gamma, uo, ui, fs);
          for (int v = 0; v < m.nv; ++v) vol[v] -= fs[v] / w[0];
        }
        for (int v = 0; v < m.nv; ++v) acc[v] -= ((real)2.0 / (real)m.h[dir]) * vol[v];
      }
      for (int v = 0; v < m.nv; ++v) du[(e * m.nv + v) * m.P + node] = acc[v];
    }
  }
  return 0;
}

#ifdef OR_CSTEP
/* Jacobian-vector product J(u) v of the rhs by complex-step differentiation:
 * J v = Im(rhs(u + i eps v)) / eps, exact to rounding for eps = 1e-30 since
 * no difference of nearby values is taken. Same element selection as or_rhs
 * (jv written for the listed elements). */
int or_rhs_jvp(int d, int N, const int *n, const double *dom, double gamma, int vflux, int sflux,
               const double *u, const double *vdir, double *jv, const long long *elems,
               long long n_elems, int nthreads) {
  mesh_t m;
  if (mesh_init(&m, d, N, n, dom)) return -1;
  long long nvals = m.nelem * m.nv * m.P;
  const double eps = 1.0e-30;
  real *uc = (real *)malloc(sizeof(real) * nvals);
  real *dc = (real *)malloc(sizeof(real) * nvals);
  if (!uc || !dc) { free(uc); free(dc); return -2; }
  for (long long t = 0; t < nvals; ++t) { uc[t] = u[t] + I * (eps * vdir[t]); dc[t] = 0.0; }
  int rc = orc_rhs(d, N, n, dom, gamma, vflux, sflux, uc, dc, elems, n_elems, nthreads);
  for (long long t = 0; t < nvals; ++t) jv[t] = cimag(dc[t]) / eps;
  free(uc); free(dc);
  return rc;
}
#endif

#ifdef OR_COUNT
/* Operation counts of the method's pieces, from the formulas above evaluated
 * with the counting scalar (one per +, -, *, /, log1p, sqrt). */
long long or_op_count = 0;

/* one two-point flux (kind as in or_two_point) between conserved states;
 * includes the two conserved -> primitive conversions the flux makes */
extern "C" long long orn_ops_two_point(int kind, int d, int n, double gamma, const double *uL,
                                       const double *uR) {
  real a[MAXV], b[MAXV], f[MAXV];
  for (int v = 0; v < d + 2; ++v) { a[v] = uL[v]; b[v] = uR[v]; }
  or_op_count = 0;
  if (OR(two_point)(kind, d, n, gamma, a, b, f)) return -1;
  return or_op_count;
}

/* one conserved -> primitive conversion */
extern "C" long long orn_ops_cons2prim(int d, double gamma, const double *u) {
  real a[MAXV], rho, v[3], p;
  for (int k = 0; k < d + 2; ++k) a[k] = u[k];
  or_op_count = 0;
  cons2prim(d, gamma, a, &rho, v, &p);
  return or_op_count;
}

/* the whole rhs of the elements listed (all when elems is NULL), as the
 * oracle evaluates it (both orders of every pair, primitives per flux) */
extern "C" long long orn_ops_rhs(int d, int N, const int *n, const double *dom, double gamma,
                                 int vflux, int sflux, const double *u, const long long *elems,
                                 long long n_elems) {
  mesh_t m;
  if (mesh_init(&m, d, N, n, dom)) return -1;
  long long nv = m.nelem * m.nv * m.P;
  real *uc = new real[nv], *dc = new real[nv];
  for (long long t = 0; t < nv; ++t) uc[t] = u[t];
  or_op_count = 0;
  int rc = OR(rhs)(d, N, n, dom, gamma, vflux, sflux, uc, dc, elems, n_elems, 1);
  long long ops = or_op_count;
  delete[] uc;
  delete[] dc;
  return rc ? -1 : ops;
}
#endif

#if !defined(OR_CSTEP) && !defined(OR_LONGDOUBLE) && !defined(OR_COUNT)
/* One 2N-storage RK stage over nvals values: k <- a k + dt du; u <- u + b k. */
void or_rk_stage(long long nvals, double *u, double *k, const double *du, double a, double b,
                 double dt) {
  for (long long t = 0; t < nvals; ++t) {
    k[t] = a * k[t] + dt * du[t];
    u[t] = u[t] + b * k[t];
  }
}

/* CFL time step: dt = cfl * 2 / ((N+1) * max_e sum_dir (2/h_dir) max_nodes(|v_dir| + c)). */
double or_max_dt(int d, int N, const int *n, const double *dom, double gamma, double cfl,
                 const double *u) {
  mesh_t m;
  if (mesh_init(&m, d, N, n, dom)) return -1.0;
  double worst = 0.0;
  for (long long e = 0; e < m.nelem; ++e) {
    double lam[3] = {0.0, 0.0, 0.0};
    for (long long node = 0; node < m.P; ++node) {
      double un[MAXV], rho, v[3], p;
      load_node(&m, u, e, node, un);
      cons2prim(d, gamma, un, &rho, v, &p);
      double c = sqrt(gamma * p / rho);
      for (int k = 0; k < d; ++k) {
        double s = fabs(v[k]) + c;
        if (s > lam[k]) lam[k] = s;
      }
    }
    double sum = 0.0;
    for (int k = 0; k < d; ++k) sum += (2.0 / m.h[k]) * lam[k];
    if (sum > worst) worst = sum;
  }
  return cfl * 2.0 / ((N + 1) * worst);
}

/* Neumaier-compensated accumulation. */
typedef struct { double s, c; } nsum_t;
static void nsum_add(nsum_t *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

/* Integrals over the domain by the LGL quadrature of each element:
 * out = [rho, rho v_1..rho v_d, E, S, K] with entropy S = -rho s/(gamma-1),
 * s = ln p - gamma ln rho, and kinetic energy K = rho |v|^2 / 2
 * (d + 4 values). Compensated (Neumaier) sums. */
int or_integrals(int d, int N, const int *n, const double *dom, double gamma, const double *u,
                 double *out) {
  mesh_t m;
  if (mesh_init(&m, d, N, n, dom)) return -1;
  double xi[16], w[16];
  or_lgl(N, xi, w);
  double jac = 1.0;
  for (int k = 0; k < d; ++k) jac *= 0.5 * m.h[k];
  int nq = d + 4;
  nsum_t acc[7];
  memset(acc, 0, sizeof(acc));
  for (long long e = 0; e < m.nelem; ++e) {
    for (long long node = 0; node < m.P; ++node) {
      double un[MAXV], rho, v[3], p;
      load_node(&m, u, e, node, un);
      cons2prim(d, gamma, un, &rho, v, &p);
      double wq = jac;
      for (int k = 0; k < d; ++k) wq *= w[node_coord(&m, node, k)];
      double v2 = 0.0;
      for (int k = 0; k < d; ++k) v2 += v[k] * v[k];
      double q[7];
      for (int v2i = 0; v2i < m.nv; ++v2i) q[v2i] = un[v2i];
      q[m.nv] = -rho * (log(p) - gamma * log(rho)) / (gamma - 1.0);
      q[m.nv + 1] = 0.5 * rho * v2;
      for (int k = 0; k < nq; ++k) nsum_add(&acc[k], wq * q[k]);
    }
  }
  for (int k = 0; k < nq; ++k) out[k] = acc[k].s + acc[k].c;
  return 0;
}
#endif
