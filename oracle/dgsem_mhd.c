/*
 * Plain FP64 CPU oracle of the DGSEM right-hand side for the 3D ideal
 * magnetohydrodynamics (MHD) equations on a uniform periodic Cartesian mesh.
 *
 * TEST INFRASTRUCTURE ONLY, like dgsem_oracle.c (whose basis routines it
 * calls): only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it; it shares nothing with the CUDA library.
 *
 * What it follows (paper: "Adaptive numerical simulations with Trixi.jl"):
 *   - Sec. 3.1 runs the 3D ideal MHD equations (Alfven wave propagation)
 *     with a weak-form solver and notes that the MHD discretisations need
 *     non-conservative terms; the weak form is the split form with the
 *     central volume flux (Sec. 3.1, gassner2016split);
 *   - ideal MHD, u = (rho, rho v, E, B), E = p/(gamma-1) + rho|v|^2/2 +
 *     |B|^2/2, flux in direction n:
 *       (rho v_n, rho v_n v + (p + |B|^2/2) e_n - B_n B,
 *        v_n (E + p + |B|^2/2) - B_n (v.B), v_n B - B_n v);
 *   - the non-conservative (Powell) term -(div B) Phi(u),
 *     Phi = (0, B, v.B, v), with div B discretised like the flux divergence:
 *     the split form with the central two-point value (B_i + B_m)/2 and the
 *     interface average of the two traces (this equals the nodal derivative
 *     of the interpolant plus the SBP correction toward the interface
 *     average);
 *   - local Lax-Friedrichs at the faces with lambda = max(|v_n,L|, |v_n,R|) +
 *     max(c_f,L, c_f,R), c_f the fast magnetosonic speed in direction n:
 *       c_f^2 = (a^2 + b^2 + sqrt((a^2 + b^2)^2 - 4 a^2 b_n^2)) / 2,
 *       a^2 = gamma p / rho, b^2 = |B|^2 / rho, b_n^2 = B_n^2 / rho;
 *     or HLL (the weak-form runs of Sec. 3.1 couple elements with HLL) with
 *     the signal speeds S_L = min(v_n,L - c_f,L, v_n,R - c_f,R), S_R =
 *     max(v_n,L + c_f,L, v_n,R + c_f,R).
 *   - flux differencing with an entropy-conservative (EC) two-point flux in
 *     the volume and at the faces (the paper's second MHD solver, Sec. 3.1,
 *     whose EC flux it cites without formulas; the non-conservative term
 *     keeps the split form above). With beta = rho/(2p), entropy variables
 *     w = ((gamma - s)/(gamma-1) - beta|v|^2, 2 beta v, -2 beta, 2 beta B),
 *     theta = w . Phi = 2 beta v.B and psi_n = rho v_n + beta v_n |B|^2, a
 *     two-point flux f# makes the scheme entropy conservative when
 *       [[w]] . f# + {B_n} [[theta]] = [[psi_n]]
 *     ({a} the mean, [[a]] the jump). Splitting every jump of a product
 *     into means times jumps ([[psi_n]] grouped as {beta |B|^2} [[v_n]] +
 *     {v_n} [[beta |B|^2]]) and matching the jumps of rho, beta, v and B
 *     gives the flux of or_mhd_flux_ec below.
 * Readings (the paper gives no formulas): the weak form with the Powell
 * term in this form, the LLF wave speed, this EC flux, the Alfven wave of
 * the tests.
 *
 * du_i = -(2/h) sum_dir [ sum_m Dt_im f#(u_i, u_m) + delta_iN F*_R/w_N
 *                          - delta_i0 F*_L/w_0 ]
 *        - Phi(u_i) (2/h) sum_dir [ sum_m Dt_im (B_i + B_m)/2 + delta_iN {B}_R/w_N
 *                                   - delta_i0 {B}_L/w_0 ]
 * (B = B_dir, {B} the average of the two traces), f# the central flux, each
 * pair evaluated for the node it updates, every face value once per
 * adjacent element.
 */
#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_dtilde(int N, double *Dt, double *w);
double or_ln_mean(double x, double y);

#define MV 8
#define NPMAX 16

/* primitive (rho, v, p) of an MHD state */
static void mhd_prim(double gamma, const double *u, double *rho, double *v, double *p) {
  *rho = u[0];
  for (int k = 0; k < 3; ++k) v[k] = u[1 + k] / u[0];
  const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  const double b2 = u[5] * u[5] + u[6] * u[6] + u[7] * u[7];
  *p = (gamma - 1.0) * (u[4] - 0.5 * u[0] * v2 - 0.5 * b2);
}

/* physical flux in direction n */
void or_mhd_flux(int n, double gamma, const double *u, double *f) {
  double rho, v[3], p;
  mhd_prim(gamma, u, &rho, v, &p);
  const double *B = u + 5;
  const double b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
  const double vb = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
  const double pt = p + 0.5 * b2;
  f[0] = rho * v[n];
  for (int k = 0; k < 3; ++k) f[1 + k] = rho * v[n] * v[k] - B[n] * B[k];
  f[1 + n] += pt;
  f[4] = v[n] * (u[4] + pt) - B[n] * vb;
  for (int k = 0; k < 3; ++k) f[5 + k] = v[n] * B[k] - B[n] * v[k];
}

/* fast magnetosonic speed in direction n */
double or_mhd_fast_speed(int n, double gamma, const double *u) {
  double rho, v[3], p;
  mhd_prim(gamma, u, &rho, v, &p);
  const double *B = u + 5;
  const double a2 = gamma * p / rho;
  const double b2 = (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho;
  const double bn2 = B[n] * B[n] / rho;
  const double s = a2 + b2;
  return sqrt(0.5 * (s + sqrt(s * s - 4.0 * a2 * bn2)));
}

/* local Lax-Friedrichs flux in direction n */
void or_mhd_llf(int n, double gamma, const double *uL, const double *uR, double *f) {
  double fL[MV], fR[MV];
  or_mhd_flux(n, gamma, uL, fL);
  or_mhd_flux(n, gamma, uR, fR);
  const double vL = uL[1 + n] / uL[0], vR = uR[1 + n] / uR[0];
  const double lam = fmax(fabs(vL), fabs(vR)) +
                     fmax(or_mhd_fast_speed(n, gamma, uL), or_mhd_fast_speed(n, gamma, uR));
  for (int v = 0; v < MV; ++v) f[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

/* Entropy-conservative two-point flux in direction n (derivation in the
 * header): with rho_ln, beta_ln the logarithmic means and {.} arithmetic
 * means,
 *   f_rho = rho_ln {v_n}
 *   f_m   = f_rho {v} - {B_n} {B} + ({rho} + {beta |B|^2}) / (2 {beta}) e_n
 *   f_B   = {v_n} {B} - {B_n} {v}            (zero in component n)
 *   f_E   = f_rho (1/(2 (gamma-1) beta_ln) - {|v|^2}/2) + f_m . {v}
 *           + f_B . {B} - {v_n} {|B|^2}/2 + {B_n} {v.B} */
void or_mhd_flux_ec(int n, double gamma, const double *uL, const double *uR, double *f) {
  double rL, vL[3], pL, rR, vR[3], pR;
  mhd_prim(gamma, uL, &rL, vL, &pL);
  mhd_prim(gamma, uR, &rR, vR, &pR);
  const double *BL = uL + 5, *BR = uR + 5;
  const double bL = rL / (2.0 * pL), bR = rR / (2.0 * pR);
  double va[3], Ba[3], v2 = 0.0, B2 = 0.0, vB = 0.0, bB2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    va[k] = 0.5 * (vL[k] + vR[k]);
    Ba[k] = 0.5 * (BL[k] + BR[k]);
    v2 += 0.5 * (vL[k] * vL[k] + vR[k] * vR[k]);
    B2 += 0.5 * (BL[k] * BL[k] + BR[k] * BR[k]);
    vB += 0.5 * (vL[k] * BL[k] + vR[k] * BR[k]);
    bB2 += 0.5 * (bL * BL[k] * BL[k] + bR * BR[k] * BR[k]);
  }
  const double rho_ln = or_ln_mean(rL, rR), beta_ln = or_ln_mean(bL, bR);
  const double ra = 0.5 * (rL + rR), ba = 0.5 * (bL + bR);
  f[0] = rho_ln * va[n];
  for (int k = 0; k < 3; ++k) f[1 + k] = f[0] * va[k] - Ba[n] * Ba[k];
  f[1 + n] += (ra + bB2) / (2.0 * ba);
  for (int k = 0; k < 3; ++k) f[5 + k] = va[n] * Ba[k] - Ba[n] * va[k];
  double fmv = 0.0, fBB = 0.0;
  for (int k = 0; k < 3; ++k) {
    fmv += f[1 + k] * va[k];
    fBB += f[5 + k] * Ba[k];
  }
  f[4] = f[0] * (1.0 / (2.0 * (gamma - 1.0) * beta_ln) - 0.5 * v2) + fmv + fBB - 0.5 * va[n] * B2 +
         Ba[n] * vB;
}

/* HLL flux in direction n: f(u_L) if S_L >= 0, f(u_R) if S_R <= 0, else
 * (S_R f_L - S_L f_R + S_L S_R (u_R - u_L)) / (S_R - S_L). */
void or_mhd_hll(int n, double gamma, const double *uL, const double *uR, double *f) {
  double fL[MV], fR[MV];
  or_mhd_flux(n, gamma, uL, fL);
  or_mhd_flux(n, gamma, uR, fR);
  const double vL = uL[1 + n] / uL[0], vR = uR[1 + n] / uR[0];
  const double cL = or_mhd_fast_speed(n, gamma, uL), cR = or_mhd_fast_speed(n, gamma, uR);
  const double sL = fmin(vL - cL, vR - cR), sR = fmax(vL + cL, vR + cR);
  for (int v = 0; v < MV; ++v) {
    if (sL >= 0.0) f[v] = fL[v];
    else if (sR <= 0.0) f[v] = fR[v];
    else f[v] = (sR * fL[v] - sL * fR[v] + sL * sR * (uR[v] - uL[v])) / (sR - sL);
  }
}

/* surface flux ids of or_mhd_rhs: 0 LLF, 1 HLL, 2 EC */
static void mhd_surface(int sflux, int n, double gamma, const double *uL, const double *uR,
                        double *f) {
  if (sflux == 1) or_mhd_hll(n, gamma, uL, uR, f);
  else if (sflux == 2) or_mhd_flux_ec(n, gamma, uL, uR, f);
  else or_mhd_llf(n, gamma, uL, uR, f);
}

/* volume two-point flux ids of or_mhd_rhs: 0 central (the weak form), 1 EC */
static void mhd_volume(int vflux, int n, double gamma, const double *ui, const double *um,
                       double *f) {
  if (vflux == 1) {
    or_mhd_flux_ec(n, gamma, ui, um, f);
  } else {
    double fi[MV], fm[MV];
    or_mhd_flux(n, gamma, ui, fi);
    or_mhd_flux(n, gamma, um, fm);
    for (int v = 0; v < MV; ++v) f[v] = 0.5 * (fi[v] + fm[v]);
  }
}

typedef struct {
  int N, np;
  int n[3];
  double h[3];
  long long nelem, P;
} mmesh_t;

static int mmesh_init(mmesh_t *m, int N, const int *n, const double *dom) {
  if (N < 1 || N > 15) return -1;
  m->N = N;
  m->np = N + 1;
  m->nelem = 1;
  for (int k = 0; k < 3; ++k) {
    if (n[k] < 1 || !(dom[2 * k + 1] > dom[2 * k])) return -1;
    m->n[k] = n[k];
    m->h[k] = (dom[2 * k + 1] - dom[2 * k]) / n[k];
    m->nelem *= n[k];
  }
  m->P = (long long)m->np * m->np * m->np;
  return 0;
}

static long long m_with(const mmesh_t *m, long long node, int r, int a) {
  int c[3] = {(int)(node % m->np), (int)((node / m->np) % m->np),
              (int)(node / ((long long)m->np * m->np))};
  c[r] = a;
  return c[0] + (long long)m->np * (c[1] + (long long)m->np * c[2]);
}

static int m_coord(const mmesh_t *m, long long node, int r) {
  long long q = node;
  for (int k = 0; k < r; ++k) q /= m->np;
  return (int)(q % m->np);
}

static long long m_neighbour(const mmesh_t *m, long long e, int r, int s) {
  int c[3] = {(int)(e % m->n[0]), (int)((e / m->n[0]) % m->n[1]),
              (int)(e / ((long long)m->n[0] * m->n[1]))};
  c[r] = (c[r] + s + m->n[r]) % m->n[r];
  return c[0] + (long long)m->n[0] * (c[1] + (long long)m->n[1] * c[2]);
}

static void m_load(const mmesh_t *m, const double *u, long long e, long long node, double *out) {
  for (int v = 0; v < MV; ++v) out[v] = u[(e * MV + v) * m->P + node];
}

/* du = rhs(u) for the listed elements (all when elems is NULL); powell = 0
 * drops the non-conservative term; vflux 0 central (weak form), 1 EC;
 * sflux 0 LLF, 1 HLL, 2 EC. Returns 0 or -1 on bad arguments. */
int or_mhd_rhs(int N, const int *n, const double *dom, double gamma, int powell, int vflux,
               int sflux, const double *u, double *du, const long long *elems, long long n_elems,
               int nthreads) {
  mmesh_t m;
  if (mmesh_init(&m, N, n, dom) || vflux < 0 || vflux > 1 || sflux < 0 || sflux > 2) return -1;
  double Dt[NPMAX * NPMAX], w[NPMAX];
  or_dtilde(N, Dt, w);
  const long long count = elems ? n_elems : m.nelem;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (long long s = 0; s < count; ++s) {
    const long long e = elems ? elems[s] : s;
    for (long long node = 0; node < m.P; ++node) {
      double ui[MV], acc[MV], divb = 0.0;
      m_load(&m, u, e, node, ui);
      for (int v = 0; v < MV; ++v) acc[v] = 0.0;
      for (int r = 0; r < 3; ++r) {
        const int i = m_coord(&m, node, r);
        double vol[MV], db = 0.0;
        for (int v = 0; v < MV; ++v) vol[v] = 0.0;
        for (int a = 0; a <= N; ++a) {
          double um[MV], fp[MV];
          m_load(&m, u, e, m_with(&m, node, r, a), um);
          mhd_volume(vflux, r, gamma, ui, um, fp);
          for (int v = 0; v < MV; ++v) vol[v] += Dt[i * m.np + a] * fp[v];
          db += Dt[i * m.np + a] * (0.5 * (ui[5 + r] + um[5 + r]));
        }
        if (i == N) {
          double uo[MV], fs[MV];
          m_load(&m, u, m_neighbour(&m, e, r, +1), m_with(&m, node, r, 0), uo);
          mhd_surface(sflux, r, gamma, ui, uo, fs);
          for (int v = 0; v < MV; ++v) vol[v] += fs[v] / w[N];
          db += 0.5 * (ui[5 + r] + uo[5 + r]) / w[N];
        }
        if (i == 0) {
          double uo[MV], fs[MV];
          m_load(&m, u, m_neighbour(&m, e, r, -1), m_with(&m, node, r, N), uo);
          mhd_surface(sflux, r, gamma, uo, ui, fs);
          for (int v = 0; v < MV; ++v) vol[v] -= fs[v] / w[0];
          db -= 0.5 * (uo[5 + r] + ui[5 + r]) / w[0];
        }
        for (int v = 0; v < MV; ++v) acc[v] -= (2.0 / m.h[r]) * vol[v];
        divb += (2.0 / m.h[r]) * db;
      }
      if (powell) {
        double rho, v[3], p;
        mhd_prim(gamma, ui, &rho, v, &p);
        const double *B = ui + 5;
        const double phi[MV] = {0.0, B[0], B[1], B[2], v[0] * B[0] + v[1] * B[1] + v[2] * B[2],
                                v[0], v[1], v[2]};
        for (int q = 0; q < MV; ++q) acc[q] -= phi[q] * divb;
      }
      for (int v = 0; v < MV; ++v) du[(e * MV + v) * m.P + node] = acc[v];
    }
  }
  return 0;
}

/* CFL time step: dt = cfl 2 / ((N+1) max_e sum_dir (2/h_dir) max_nodes(|v_dir| + c_f,dir)). */
double or_mhd_max_dt(int N, const int *n, const double *dom, double gamma, double cfl,
                     const double *u) {
  mmesh_t m;
  if (mmesh_init(&m, N, n, dom)) return -1.0;
  double worst = 0.0;
  for (long long e = 0; e < m.nelem; ++e) {
    double lam[3] = {0.0, 0.0, 0.0};
    for (long long node = 0; node < m.P; ++node) {
      double un[MV];
      m_load(&m, u, e, node, un);
      for (int r = 0; r < 3; ++r) {
        const double s = fabs(un[1 + r] / un[0]) + or_mhd_fast_speed(r, gamma, un);
        if (s > lam[r]) lam[r] = s;
      }
    }
    double sum = 0.0;
    for (int r = 0; r < 3; ++r) sum += (2.0 / m.h[r]) * lam[r];
    if (sum > worst) worst = sum;
  }
  return cfl * 2.0 / ((N + 1) * worst);
}

/* ---- the warped periodic box of the paper's performance runs (Sec. 3.1) ----
 * The same operators on the curvilinear mesh of dgsem_curved.c (geometry:
 * metric terms Ja[e][r][d][P] = (J a^r)_d and Jacobians J[e][P] from
 * or_curved_geometry): in direction r the two-point flux is taken along the
 * mean of the two nodes' metric vectors, sum_d g_d f#_d, the face flux along
 * the metric vector of the left element's face node (LLF and HLL in the unit
 * direction, scaled by its length), the Powell divergence as
 * (1/J) sum_r [sum_m Dt_im g_im . (B_i + B_m)/2 + face terms with
 * {B} . g], and du = -(1/J) (...) - Phi (div B). */

/* fast magnetosonic speed in the unit direction nh */
static double mhd_fast_speed_dir(double gamma, const double *nh, const double *u) {
  double rho, v[3], p;
  mhd_prim(gamma, u, &rho, v, &p);
  const double *B = u + 5;
  const double a2 = gamma * p / rho;
  const double b2 = (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho;
  const double bn = B[0] * nh[0] + B[1] * nh[1] + B[2] * nh[2];
  const double bn2 = bn * bn / rho;
  const double s = a2 + b2;
  return sqrt(0.5 * (s + sqrt(s * s - 4.0 * a2 * bn2)));
}

/* sum_d g_d f_d(u) */
static void mhd_flux_dir(double gamma, const double *g, const double *u, double *f) {
  double fd[MV];
  for (int v = 0; v < MV; ++v) f[v] = 0.0;
  for (int d = 0; d < 3; ++d) {
    or_mhd_flux(d, gamma, u, fd);
    for (int v = 0; v < MV; ++v) f[v] += g[d] * fd[v];
  }
}

/* two-point volume flux along g: central or EC (sum_d g_d f#_d) */
static void mhd_volume_dir(int vflux, double gamma, const double *g, const double *ui,
                           const double *um, double *f) {
  if (vflux == 1) {
    double fd[MV];
    for (int v = 0; v < MV; ++v) f[v] = 0.0;
    for (int d = 0; d < 3; ++d) {
      or_mhd_flux_ec(d, gamma, ui, um, fd);
      for (int v = 0; v < MV; ++v) f[v] += g[d] * fd[v];
    }
    return;
  }
  double fi[MV], fm[MV];
  mhd_flux_dir(gamma, g, ui, fi);
  mhd_flux_dir(gamma, g, um, fm);
  for (int v = 0; v < MV; ++v) f[v] = 0.5 * (fi[v] + fm[v]);
}

/* face flux along the (non-normalised) metric vector g: 0 LLF, 1 HLL (in the
 * unit direction, scaled by |g|), 2 EC */
static void mhd_surface_dir(int sflux, double gamma, const double *g, const double *uL,
                            const double *uR, double *f) {
  if (sflux == 2) {
    mhd_volume_dir(1, gamma, g, uL, uR, f);
    return;
  }
  const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  const double nh[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
  double fl[MV], fr[MV];
  mhd_flux_dir(gamma, g, uL, fl);
  mhd_flux_dir(gamma, g, uR, fr);
  const double vl = (uL[1] * nh[0] + uL[2] * nh[1] + uL[3] * nh[2]) / uL[0];
  const double vr = (uR[1] * nh[0] + uR[2] * nh[1] + uR[3] * nh[2]) / uR[0];
  const double cl = mhd_fast_speed_dir(gamma, nh, uL), cr = mhd_fast_speed_dir(gamma, nh, uR);
  if (sflux == 0) {
    const double lam = fmax(fabs(vl), fabs(vr)) + fmax(cl, cr);
    for (int v = 0; v < MV; ++v) f[v] = 0.5 * (fl[v] + fr[v]) - 0.5 * lam * gn * (uR[v] - uL[v]);
    return;
  }
  const double sL = fmin(vl - cl, vr - cr), sR = fmax(vl + cl, vr + cr);
  for (int v = 0; v < MV; ++v) {
    if (sL >= 0.0) f[v] = fl[v];
    else if (sR <= 0.0) f[v] = fr[v];
    else f[v] = (sR * fl[v] - sL * fr[v] + sL * sR * gn * (uR[v] - uL[v])) / (sR - sL);
  }
}

static void mhd_metric(const mmesh_t *m, const double *Ja, long long e, int r, long long node,
                       double *g) {
  for (int d = 0; d < 3; ++d) g[d] = Ja[((e * 3 + r) * 3 + d) * m->P + node];
}

/* du = rhs(u) on the warped box with geometry (Ja, J) of or_curved_geometry
 * (elements_per_dim n, degree N), for the listed elements (all when elems is
 * NULL). Flux ids as in or_mhd_rhs. Returns 0 or -1 on bad arguments. */
int or_mhd_curved_rhs(int N, const int *n, double gamma, int powell, int vflux, int sflux,
                      const double *Ja, const double *J, const double *u, double *du,
                      const long long *elems, long long n_elems, int nthreads) {
  mmesh_t m;
  const double box[6] = {-1.0, 1.0, -1.0, 1.0, -1.0, 1.0};
  if (mmesh_init(&m, N, n, box) || vflux < 0 || vflux > 1 || sflux < 0 || sflux > 2) return -1;
  double Dt[NPMAX * NPMAX], w[NPMAX];
  or_dtilde(N, Dt, w);
  const long long count = elems ? n_elems : m.nelem;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (long long s = 0; s < count; ++s) {
    const long long e = elems ? elems[s] : s;
    for (long long node = 0; node < m.P; ++node) {
      double ui[MV], acc[MV], db = 0.0;
      m_load(&m, u, e, node, ui);
      for (int v = 0; v < MV; ++v) acc[v] = 0.0;
      for (int r = 0; r < 3; ++r) {
        const int i = m_coord(&m, node, r);
        double gi[3];
        mhd_metric(&m, Ja, e, r, node, gi);
        for (int a = 0; a <= N; ++a) {
          const long long nm = m_with(&m, node, r, a);
          double um[MV], gm[3], g[3], f[MV];
          m_load(&m, u, e, nm, um);
          mhd_metric(&m, Ja, e, r, nm, gm);
          for (int k = 0; k < 3; ++k) g[k] = 0.5 * (gi[k] + gm[k]);
          mhd_volume_dir(vflux, gamma, g, ui, um, f);
          for (int v = 0; v < MV; ++v) acc[v] += Dt[i * m.np + a] * f[v];
          double bg = 0.0;
          for (int k = 0; k < 3; ++k) bg += g[k] * 0.5 * (ui[5 + k] + um[5 + k]);
          db += Dt[i * m.np + a] * bg;
        }
        if (i == N) {
          double uo[MV], f[MV], bg = 0.0;
          m_load(&m, u, m_neighbour(&m, e, r, +1), m_with(&m, node, r, 0), uo);
          mhd_surface_dir(sflux, gamma, gi, ui, uo, f);
          for (int v = 0; v < MV; ++v) acc[v] += f[v] / w[N];
          for (int k = 0; k < 3; ++k) bg += gi[k] * 0.5 * (ui[5 + k] + uo[5 + k]);
          db += bg / w[N];
        }
        if (i == 0) {
          const long long el = m_neighbour(&m, e, r, -1), nl = m_with(&m, node, r, N);
          double uo[MV], gl[3], f[MV], bg = 0.0;
          m_load(&m, u, el, nl, uo);
          mhd_metric(&m, Ja, el, r, nl, gl);
          mhd_surface_dir(sflux, gamma, gl, uo, ui, f);
          for (int v = 0; v < MV; ++v) acc[v] -= f[v] / w[0];
          for (int k = 0; k < 3; ++k) bg += gl[k] * 0.5 * (uo[5 + k] + ui[5 + k]);
          db -= bg / w[0];
        }
      }
      const double Jn = J[e * m.P + node];
      double phi[MV] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      if (powell) {
        double rho, v[3], p;
        mhd_prim(gamma, ui, &rho, v, &p);
        const double *B = ui + 5;
        phi[1] = B[0];
        phi[2] = B[1];
        phi[3] = B[2];
        phi[4] = v[0] * B[0] + v[1] * B[1] + v[2] * B[2];
        phi[5] = v[0];
        phi[6] = v[1];
        phi[7] = v[2];
      }
      for (int v = 0; v < MV; ++v) du[(e * MV + v) * m.P + node] = -(acc[v] + phi[v] * db) / Jn;
    }
  }
  return 0;
}

/* CFL time step on the warped box: dt = cfl 2 / ((N+1) max_e sum_r lam_r),
 * lam_r = max over the element's nodes of (|v . J a^r| + c_f(a^r) |J a^r|) / J. */
double or_mhd_curved_max_dt(int N, const int *n, double gamma, double cfl, const double *Ja,
                            const double *J, const double *u) {
  mmesh_t m;
  const double box[6] = {-1.0, 1.0, -1.0, 1.0, -1.0, 1.0};
  if (mmesh_init(&m, N, n, box)) return -1.0;
  double worst = 0.0;
  for (long long e = 0; e < m.nelem; ++e) {
    double lam[3] = {0.0, 0.0, 0.0};
    for (long long node = 0; node < m.P; ++node) {
      double un[MV];
      m_load(&m, u, e, node, un);
      for (int r = 0; r < 3; ++r) {
        double g[3];
        mhd_metric(&m, Ja, e, r, node, g);
        const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const double nh[3] = {g[0] / gn, g[1] / gn, g[2] / gn};
        const double vg = (un[1] * g[0] + un[2] * g[1] + un[3] * g[2]) / un[0];
        const double s = (fabs(vg) + mhd_fast_speed_dir(gamma, nh, un) * gn) / J[e * m.P + node];
        if (s > lam[r]) lam[r] = s;
      }
    }
    const double sum = lam[0] + lam[1] + lam[2];
    if (sum > worst) worst = sum;
  }
  return cfl * 2.0 / ((N + 1) * worst);
}
