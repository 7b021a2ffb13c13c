/*
 * Plain FP64 CPU oracle of the DGSEM right-hand side on the curvilinear
 * (warped) periodic hexahedral mesh of the paper's performance benchmark,
 * for the 3D compressible Euler equations, with optional manufactured-
 * solution source terms.
 *
 * TEST INFRASTRUCTURE ONLY, like dgsem_oracle.c (whose exported flux and
 * basis routines it calls): only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py use it; it shares nothing with
 * the CUDA library.
 *
 * What it follows (paper: "Adaptive numerical simulations with Trixi.jl"):
 *   - Sec. 3.1 (setup of the performance comparison): a periodic box
 *     [-1,1]^3 of n^3 elements whose interior is warped by the mapping of
 *     that section (adapted from chan2019efficient), the 3D compressible
 *     Euler equations with a manufactured solution, a weak-form solver with
 *     HLL surface flux and a flux-differencing solver with an
 *     entropy-conservative flux in the volume and at the surface;
 *   - the curvilinear DGSEM of the cited texts (Kopriva 2009): each element
 *     is the image of the reference cube under a polynomial of degree N
 *     interpolating the mapping at the LGL nodes; the metric terms J a^i are
 *     computed in the conservative curl form (Kopriva 2006),
 *         (J a^i)_n = -e_i . curl_xi( I^N( X_l grad_xi X_m ) ),  (n, m, l) cyclic,
 *     which makes sum_i d/dxi^i (J a^i)_n = 0 hold discretely (free-stream
 *     preservation), and J = a_1 . (a_2 x a_3) with a_r = dX/dxi^r;
 *   - the split-form flux differencing on curved elements: for reference
 *     direction r,
 *         du_i = -(1/J_i) sum_r [ sum_m Dt_im F#^r(u_i, u_m)
 *                                + delta_iN F*^r_R / w_N - delta_i0 F*^r_L / w_0 ] + S_i,
 *     F#^r(a, b) = sum_n (J a^r_n(a) + J a^r_n(b))/2 f#_n(u_a, u_b) (the
 *     contravariant two-point flux with averaged metric terms), and at a
 *     face F*^r = the surface flux in the direction of the metric vector
 *     J a^r of the face node, taken from the element on the left of the face
 *     (reading: one flux per face, as in the Cartesian oracle);
 *   - the Cartesian special case (no warping): J a^r = (h/2)^2 e_r,
 *     J = (h/2)^3, which gives back the Cartesian operator of dgsem_oracle.c.
 * The manufactured solution (a reading: the paper names one but gives no
 * formula) is rho = 2 + A sin(pi (x + y + z - t)), v = (1, 1, 1), E = rho^2,
 * A = 0.1; its source term S = d_t u + div F(u) is written out in
 * or_manufactured_source.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* from dgsem_oracle.c (double build) */
int or_lgl(int N, double *xi, double *w);
int or_diff_matrix(int N, const double *xi, double *D);
int or_dtilde(int N, double *Dt, double *w);
int or_two_point(int kind, int d, int n, double gamma, const double *uL, const double *uR,
                 double *f);

#define NV 5
#define NPMAX 16

static const double kPi = 3.14159265358979323846;

/* The warping of Sec. 3.1: Cartesian reference coordinates c = (xi, eta,
 * zeta) of the box to physical (x, y, z); y first, then x (using y), then z
 * (using x and y). */
static void warp_map(double a, const double *c, double *X) {
  const double y = c[1] + a * cos(1.5 * kPi * c[0]) * cos(0.5 * kPi * c[1]) * cos(0.5 * kPi * c[2]);
  const double x = c[0] + a * cos(0.5 * kPi * c[0]) * cos(2.0 * kPi * y) * cos(0.5 * kPi * c[2]);
  const double z = c[2] + a * cos(0.5 * kPi * x) * cos(kPi * y) * cos(0.5 * kPi * c[2]);
  X[0] = x;
  X[1] = y;
  X[2] = z;
}

typedef struct {
  int N, np;
  int n[3];
  long long nelem, P;
} cmesh_t;

static int cmesh_init(cmesh_t *m, int N, const int *n) {
  if (N < 1 || N > 15) return -1;
  m->N = N;
  m->np = N + 1;
  m->nelem = 1;
  for (int k = 0; k < 3; ++k) {
    if (n[k] < 1) return -1;
    m->n[k] = n[k];
    m->nelem *= n[k];
  }
  m->P = (long long)m->np * m->np * m->np;
  return 0;
}

/* node index of (i, j, k), i (x) fastest */
static long long nidx(const cmesh_t *m, int i, int j, int k) {
  return i + (long long)m->np * (j + (long long)m->np * k);
}

static void ncoords(const cmesh_t *m, long long node, int *c) {
  c[0] = (int)(node % m->np);
  c[1] = (int)((node / m->np) % m->np);
  c[2] = (int)(node / ((long long)m->np * m->np));
}

static long long with_coord(const cmesh_t *m, long long node, int r, int a) {
  int c[3];
  ncoords(m, node, c);
  c[r] = a;
  return nidx(m, c[0], c[1], c[2]);
}

static void ecoords(const cmesh_t *m, long long e, int *c) {
  c[0] = (int)(e % m->n[0]);
  c[1] = (int)((e / m->n[0]) % m->n[1]);
  c[2] = (int)(e / ((long long)m->n[0] * m->n[1]));
}

static long long eneighbour(const cmesh_t *m, long long e, int r, int s) {
  int c[3];
  ecoords(m, e, c);
  c[r] = (c[r] + s + m->n[r]) % m->n[r];
  return c[0] + (long long)m->n[0] * (c[1] + (long long)m->n[1] * c[2]);
}

/* derivative along reference direction r of nodal values g (one element) */
static double dref(const cmesh_t *m, const double *D, const double *g, long long node, int r) {
  int c[3];
  ncoords(m, node, c);
  double s = 0.0;
  for (int a = 0; a <= m->N; ++a) s += D[c[r] * m->np + a] * g[with_coord(m, node, r, a)];
  return s;
}

/* Geometry of the warped periodic box [-1,1]^3 with n[0] x n[1] x n[2]
 * elements of degree N: node coordinates X[e][3][P], metric terms
 * Ja[e][r][n][P] = (J a^r)_n and Jacobians J[e][P]. warp = 0 gives the
 * uniform Cartesian mesh. Returns 0, -1 on bad arguments, -2 on allocation
 * failure. */
int or_curved_geometry(int N, const int *n, double warp, double *X, double *Ja, double *J) {
  cmesh_t m;
  if (cmesh_init(&m, N, n)) return -1;
  double xi[NPMAX], w[NPMAX], D[NPMAX * NPMAX];
  or_lgl(N, xi, w);
  or_diff_matrix(N, xi, D);
  const long long P = m.P;
  int fail = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
  for (long long e = 0; e < m.nelem; ++e) {
    double *x = (double *)malloc(sizeof(double) * 3 * P);
    double *v = (double *)malloc(sizeof(double) * 3 * P);
    if (!x || !v) {
      free(x);
      free(v);
#ifdef _OPENMP
#pragma omp atomic write
#endif
      fail = 1;
      continue;
    }
    int ec[3];
    ecoords(&m, e, ec);
    /* nodal values of the mapping */
    for (long long node = 0; node < P; ++node) {
      int c[3];
      ncoords(&m, node, c);
      double cart[3], Xn[3];
      for (int k = 0; k < 3; ++k) {
        const double h = 2.0 / m.n[k];
        cart[k] = -1.0 + (ec[k] + 0.5 * (xi[c[k]] + 1.0)) * h;
      }
      warp_map(warp, cart, Xn);
      for (int k = 0; k < 3; ++k) x[k * P + node] = Xn[k];
    }
    for (int k = 0; k < 3; ++k)
      memcpy(X + (e * 3 + k) * P, x + k * P, sizeof(double) * P);
    /* J = a_1 . (a_2 x a_3), a_r = dX/dxi^r */
    for (long long node = 0; node < P; ++node) {
      double a[3][3];
      for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) a[r][k] = dref(&m, D, x + k * P, node, r);
      J[e * P + node] = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) -
                        a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                        a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    }
    /* metric terms in curl form: for component n with (n, mm, l) cyclic,
     * v_b = X_l d X_mm / d xi^b at the nodes, then (J a^i)_n = -(curl v)_i */
    for (int nc = 0; nc < 3; ++nc) {
      const int mm = (nc + 1) % 3, l = (nc + 2) % 3;
      for (long long node = 0; node < P; ++node)
        for (int b = 0; b < 3; ++b)
          v[b * P + node] = x[l * P + node] * dref(&m, D, x + mm * P, node, b);
      for (long long node = 0; node < P; ++node) {
        for (int i = 0; i < 3; ++i) {
          const int a1 = (i + 1) % 3, a2 = (i + 2) % 3;
          /* (curl v)_i = d v_a2 / d xi^a1 - d v_a1 / d xi^a2 */
          const double curl = dref(&m, D, v + a2 * P, node, a1) - dref(&m, D, v + a1 * P, node, a2);
          Ja[((e * 3 + i) * 3 + nc) * P + node] = -curl;
        }
      }
    }
    free(x);
    free(v);
  }
  return fail ? -2 : 0;
}

/* Manufactured solution rho = 2 + A sin(phi), phi = pi (x + y + z - t),
 * v = (1, 1, 1), E = rho^2 (A = 0.1): the state at one point. */
void or_manufactured_state(double t, const double *X, double *u) {
  const double A = 0.1;
  const double rho = 2.0 + A * sin(kPi * (X[0] + X[1] + X[2] - t));
  u[0] = rho;
  u[1] = rho;
  u[2] = rho;
  u[3] = rho;
  u[4] = rho * rho;
}

/* Its source term S = d_t u + div F(u): with rho' = A pi cos(phi) (= d rho/dx
 * = -d rho/dt) and p = (gamma-1)(rho^2 - 3 rho / 2), p' = (gamma-1)(2 rho -
 * 3/2) rho',
 *   S = (2 rho', 2 rho' + p', 2 rho' + p', 2 rho' + p', 4 rho rho' + 3 p'). */
void or_manufactured_source(double gamma, double t, const double *X, double *S) {
  const double A = 0.1;
  const double phi = kPi * (X[0] + X[1] + X[2] - t);
  const double rho = 2.0 + A * sin(phi);
  const double drho = A * kPi * cos(phi);
  const double dp = (gamma - 1.0) * (2.0 * rho - 1.5) * drho;
  S[0] = 2.0 * drho;
  S[1] = 2.0 * drho + dp;
  S[2] = 2.0 * drho + dp;
  S[3] = 2.0 * drho + dp;
  S[4] = 4.0 * rho * drho + 3.0 * dp;
}

/* primitive (rho, v, p) and sound speed of a 3D state */
static void prim3(double gamma, const double *u, double *rho, double *v, double *p, double *c) {
  *rho = u[0];
  for (int k = 0; k < 3; ++k) v[k] = u[1 + k] / u[0];
  *p = (gamma - 1.0) * (u[4] - 0.5 * u[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
  *c = sqrt(gamma * (*p) / (*rho));
}

/* sum_n g_n F_n with F_n = a two-point flux (or the physical flux, kind 20)
 * in Cartesian direction n */
static void directed(int kind, double gamma, const double *g, const double *uL, const double *uR,
                     double *f) {
  double fn[NV];
  for (int v = 0; v < NV; ++v) f[v] = 0.0;
  for (int n = 0; n < 3; ++n) {
    or_two_point(kind, 3, n, gamma, uL, uR, fn);
    for (int v = 0; v < NV; ++v) f[v] += g[n] * fn[v];
  }
}

/* Surface flux in the direction of the (non-normalised) metric vector g:
 * 0 LLF, 2 HLL (in the unit direction g/|g|, scaled by |g|), 1 Ranocha and
 * 3 Chandrashekar (EC: sum_n g_n f#_n). */
static int surface_directed(int sflux, double gamma, const double *g, const double *uL,
                            const double *uR, double *f) {
  if (sflux == 1 || sflux == 3) {
    directed(sflux == 1 ? 0 : 1, gamma, g, uL, uR, f);
    return 0;
  }
  if (sflux != 0 && sflux != 2) return -1;
  const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  double fl[NV], fr[NV], rl, rr, vl[3], vr[3], pl, pr, cl, cr;
  directed(20, gamma, g, uL, uL, fl);
  directed(20, gamma, g, uR, uR, fr);
  prim3(gamma, uL, &rl, vl, &pl, &cl);
  prim3(gamma, uR, &rr, vr, &pr, &cr);
  const double vnl = (vl[0] * g[0] + vl[1] * g[1] + vl[2] * g[2]) / gn;
  const double vnr = (vr[0] * g[0] + vr[1] * g[1] + vr[2] * g[2]) / gn;
  if (sflux == 0) {
    const double lam = fmax(fabs(vnl), fabs(vnr)) + fmax(cl, cr);
    for (int v = 0; v < NV; ++v) f[v] = 0.5 * (fl[v] + fr[v]) - 0.5 * lam * gn * (uR[v] - uL[v]);
    return 0;
  }
  /* HLL with the Davis signal speeds in the unit direction; fl, fr are the
   * fluxes times |g|, so the result is scaled by |g| as well */
  const double sL = fmin(vnl - cl, vnr - cr), sR = fmax(vnl + cl, vnr + cr);
  for (int v = 0; v < NV; ++v) {
    if (sL >= 0.0) f[v] = fl[v];
    else if (sR <= 0.0) f[v] = fr[v];
    else f[v] = (sR * fl[v] - sL * fr[v] + sL * sR * gn * (uR[v] - uL[v])) / (sR - sL);
  }
  return 0;
}

static void load(const cmesh_t *m, const double *u, long long e, long long node, double *out) {
  for (int v = 0; v < NV; ++v) out[v] = u[(e * NV + v) * m->P + node];
}

static void metric(const cmesh_t *m, const double *Ja, long long e, int r, long long node,
                   double *g) {
  for (int n = 0; n < 3; ++n) g[n] = Ja[((e * 3 + r) * 3 + n) * m->P + node];
}

/* du = rhs(u) (+ the manufactured source at time t when source != 0) on the
 * curved mesh with geometry (Ja, J, X) from or_curved_geometry, for the listed
 * elements (all when elems is NULL). Volume flux ids 0 Ranocha,
 * 1 Chandrashekar, 2 central; surface ids 0 LLF, 1 Ranocha, 2 HLL,
 * 3 Chandrashekar. Returns 0, or -1 on bad arguments. */
int or_curved_rhs(int N, const int *n, double gamma, int vflux, int sflux, int source, double t,
                  const double *Ja, const double *J, const double *X, const double *u,
                  double *du, const long long *elems, long long n_elems, int nthreads) {
  cmesh_t m;
  if (cmesh_init(&m, N, n) || vflux < 0 || vflux > 2 || sflux < 0 || sflux > 3) return -1;
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
      double ui[NV], acc[NV];
      int c[3];
      ncoords(&m, node, c);
      load(&m, u, e, node, ui);
      for (int v = 0; v < NV; ++v) acc[v] = 0.0;
      for (int r = 0; r < 3; ++r) {
        const int i = c[r];
        double gi[3];
        metric(&m, Ja, e, r, node, gi);
        /* volume: sum_m Dt_im F#^r(u_i, u_m), averaged metric terms */
        for (int a = 0; a <= N; ++a) {
          const long long nm = with_coord(&m, node, r, a);
          double um[NV], gm[3], gavg[3], f[NV];
          load(&m, u, e, nm, um);
          metric(&m, Ja, e, r, nm, gm);
          for (int k = 0; k < 3; ++k) gavg[k] = 0.5 * (gi[k] + gm[k]);
          directed(vflux, gamma, gavg, ui, um, f);
          for (int v = 0; v < NV; ++v) acc[v] += Dt[i * m.np + a] * f[v];
        }
        /* faces: the metric vector of the left element's face node */
        if (i == N) {
          double uo[NV], f[NV];
          load(&m, u, eneighbour(&m, e, r, +1), with_coord(&m, node, r, 0), uo);
          surface_directed(sflux, gamma, gi, ui, uo, f);
          for (int v = 0; v < NV; ++v) acc[v] += f[v] / w[N];
        }
        if (i == 0) {
          const long long el = eneighbour(&m, e, r, -1), nl = with_coord(&m, node, r, N);
          double uo[NV], gl[3], f[NV];
          load(&m, u, el, nl, uo);
          metric(&m, Ja, el, r, nl, gl);
          surface_directed(sflux, gamma, gl, uo, ui, f);
          for (int v = 0; v < NV; ++v) acc[v] -= f[v] / w[0];
        }
      }
      const double Jn = J[e * m.P + node];
      double S[NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (source) {
        double Xn[3];
        for (int k = 0; k < 3; ++k) Xn[k] = X[(e * 3 + k) * m.P + node];
        or_manufactured_source(gamma, t, Xn, S);
      }
      for (int v = 0; v < NV; ++v) du[(e * NV + v) * m.P + node] = -acc[v] / Jn + S[v];
    }
  }
  return 0;
}

/* CFL time step on the curved mesh: dt = cfl 2 / ((N+1) max_e sum_r lam_r)
 * with lam_r = max over the element's nodes of (|v . J a^r| + c |J a^r|) / J,
 * the contravariant form of the Cartesian rule (equal to it without
 * warping). */
double or_curved_max_dt(int N, const int *n, double gamma, double cfl, const double *Ja,
                        const double *J, const double *u) {
  cmesh_t m;
  if (cmesh_init(&m, N, n)) return -1.0;
  double worst = 0.0;
  for (long long e = 0; e < m.nelem; ++e) {
    double lam[3] = {0.0, 0.0, 0.0};
    for (long long node = 0; node < m.P; ++node) {
      double un[NV], rho, v[3], p, c;
      load(&m, u, e, node, un);
      prim3(gamma, un, &rho, v, &p, &c);
      for (int r = 0; r < 3; ++r) {
        double g[3];
        metric(&m, Ja, e, r, node, g);
        const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const double s = (fabs(v[0] * g[0] + v[1] * g[1] + v[2] * g[2]) + c * gn) / J[e * m.P + node];
        if (s > lam[r]) lam[r] = s;
      }
    }
    const double sum = lam[0] + lam[1] + lam[2];
    if (sum > worst) worst = sum;
  }
  return cfl * 2.0 / ((N + 1) * worst);
}
