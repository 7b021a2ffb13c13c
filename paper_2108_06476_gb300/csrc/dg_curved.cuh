// Curvilinear (warped) periodic box for the 3D compressible Euler equations:
// the mesh of the paper's performance benchmark (Sec. 3.1). Each element is
// the image of the reference cube under the degree-N interpolant of the
// warping at the LGL nodes.
//
//   Geometry (once per mesh, or again for node coordinates the caller
//   gives): node coordinates X, a_r = dX/dxi^r by the
//   nodal derivative matrix, J = a_1 . (a_2 x a_3), and the metric terms in
//   the conservative curl form (J a^i)_n = -e_i . curl_xi(I^N(X_l grad X_m)),
//   (n, m, l) cyclic, which satisfy sum_i d/dxi^i (J a^i)_n = 0 discretely
//   (free-stream preservation on the curved mesh).
//   Volume: per reference direction r and node pair (a, b) of a line, the
//   contravariant two-point flux F#^r = sum_n g_n f#_n(u_a, u_b) with the
//   averaged metric vector g = ((J a^r)(a) + (J a^r)(b)) / 2; pairs once
//   (F#^r is symmetric), per-node values staged in shared memory as in the
//   Cartesian kernel.
//   Faces: the surface flux along the metric vector J a^r of the left
//   element's face node (one flux per face, face-parallel kernel).
//   Result: du = -(1/J) [sum_m Dt_im F#^r + delta_iN F*_R/w_N - delta_i0 F*_L/w_0]
//   (+ the manufactured-solution source at the stage time).
#pragma once
#include "dg_curved_decl.cuh"
#include "dg_rhs_kernels.cuh"

namespace dg {

__device__ __forceinline__ double source_time(const SourceArgs& s) {
  return *s.t0 + (s.dt ? s.c * (*s.dt) : 0.0);
}

// S = d_t u + div F(u) of the manufactured solution: with rho' = A pi cos(phi)
// and p' = (gamma-1)(2 rho - 3/2) rho',
//   S = (2 rho', 2 rho' + p' (x3), 4 rho rho' + 3 p')
__device__ __forceinline__ void manufactured_source(double x, double y, double z, double t,
                                                    double gm1, double S[5]) {
  constexpr double A = 0.1;
  double sn, cs;
  sincospi(x + y + z - t, &sn, &cs);
  const double rho = 2.0 + A * sn;
  const double drho = A * 3.14159265358979323846 * cs;
  const double dp = gm1 * (2.0 * rho - 1.5) * drho;
  S[0] = 2.0 * drho;
  S[1] = S[2] = S[3] = 2.0 * drho + dp;
  S[4] = 4.0 * rho * drho + 3.0 * dp;
}

// node with coordinate r replaced by m (3D, NP points per direction)
template <int NP>
__device__ __forceinline__ int node_with(int node, int r, int m) {
  if (r == 0) return node - node % NP + m;
  if (r == 1) return node % NP + NP * m + NP * NP * (node / (NP * NP));
  return node % (NP * NP) + NP * NP * m;
}

// ---- geometry: one CTA per element, one thread per node ----
template <int N>
__global__ void curved_geometry_kernel(CGeom cg, double* __restrict__ Ja,
                                       double* __restrict__ invJ, double* __restrict__ Jdet,
                                       double* __restrict__ X) {
  constexpr int NP = N + 1, P = NP * NP * NP;
  __shared__ double sX[3][P];
  __shared__ double sV[3][P];
  const long long e = blockIdx.x;
  const int t = threadIdx.x;
  const int c[3] = {t % NP, (t / NP) % NP, t / (NP * NP)};
  const int ec[3] = {(int)(e % cg.g.n[0]), (int)((e / cg.g.n[0]) % cg.g.n[1]),
                     (int)(e / ((long long)cg.g.n[0] * cg.g.n[1]))};
  double x, y, z;
  if (cg.Xin) {
    // node coordinates given by the caller
    x = cg.Xin[(e * 3 + 0) * P + t];
    y = cg.Xin[(e * 3 + 1) * P + t];
    z = cg.Xin[(e * 3 + 2) * P + t];
  } else {
    double cart[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double h = 2.0 / cg.g.n[k];
      cart[k] = -1.0 + (ec[k] + 0.5 * (cg.xi[c[k]] + 1.0)) * h;
    }
    // the warping of the box: y first, then x (using y), then z (using x, y)
    const double a = cg.warp;
    y = cart[1] + a * cospi(1.5 * cart[0]) * cospi(0.5 * cart[1]) * cospi(0.5 * cart[2]);
    x = cart[0] + a * cospi(0.5 * cart[0]) * cospi(2.0 * y) * cospi(0.5 * cart[2]);
    z = cart[2] + a * cospi(0.5 * x) * cospi(y) * cospi(0.5 * cart[2]);
  }
  sX[0][t] = x;
  sX[1][t] = y;
  sX[2][t] = z;
  X[(e * 3 + 0) * P + t] = x;
  X[(e * 3 + 1) * P + t] = y;
  X[(e * 3 + 2) * P + t] = z;
  __syncthreads();
  double dX[3][3];  // dX[r][k] = d X_k / d xi^r
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int m = 0; m < NP; ++m) s += cg.D[c[r]][m] * sX[k][node_with<NP>(t, r, m)];
      dX[r][k] = s;
    }
  const double J = dX[0][0] * (dX[1][1] * dX[2][2] - dX[1][2] * dX[2][1]) -
                   dX[0][1] * (dX[1][0] * dX[2][2] - dX[1][2] * dX[2][0]) +
                   dX[0][2] * (dX[1][0] * dX[2][1] - dX[1][1] * dX[2][0]);
  Jdet[e * P + t] = J;
  invJ[e * P + t] = 1.0 / J;
  for (int nc = 0; nc < 3; ++nc) {
    const int mm = (nc + 1) % 3, l = (nc + 2) % 3;
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 3; ++b) sV[b][t] = sX[l][t] * dX[b][mm];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int a1 = (i + 1) % 3, a2 = (i + 2) % 3;
      double d1 = 0.0, d2 = 0.0;
      for (int m = 0; m < NP; ++m) {
        d1 += cg.D[c[a1]][m] * sV[a2][node_with<NP>(t, a1, m)];
        d2 += cg.D[c[a2]][m] * sV[a1][node_with<NP>(t, a2, m)];
      }
      Ja[((e * 3 + i) * 3 + nc) * P + t] = -(d1 - d2);
    }
  }
}

// ---- node values staged for the volume flux (see LinePrim) ----
struct CPrim {
  double s0, s1, hp, v[3], hv[3];
};

// Ranocha's EC/KEP flux contracted with the metric vector g:
//   F0 = rho_ln (vbar . g), F_k = F0 vbar_k + pbar g_k,
//   F4 = F0 (v_L . v_R / 2 + 1/((gamma-1) ln_mean(rho/p))) + (p_L v_R.g + p_R v_L.g)/2
__device__ __forceinline__ void ranocha_contra(const CPrim& L, const CPrim& R, const double g[3],
                                               double f[5]) {
  const double rho_ln = ln_mean_halves(L.s0, R.s0);
  double vd = L.hv[0] * R.v[0];
  vd = fma(L.hv[1], R.v[1], vd);
  vd = fma(L.hv[2], R.v[2], vd);
  const double ee = add_inv_ln_mean(L.s1, R.s1, vd);
  double vb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) vb[k] = L.hv[k] + R.hv[k];
  const double vm = fma(vb[2], g[2], fma(vb[1], g[1], vb[0] * g[0]));
  const double f0 = rho_ln * vm;
  const double pb = L.hp + R.hp;
  f[0] = f0;
#pragma unroll
  for (int k = 0; k < 3; ++k) f[1 + k] = fma(f0, vb[k], pb * g[k]);
  const double vgL = fma(L.v[2], g[2], fma(L.v[1], g[1], L.v[0] * g[0]));
  const double vgR = fma(R.v[2], g[2], fma(R.v[1], g[1], R.v[0] * g[0]));
  f[4] = fma(f0, ee, fma(L.hp, vgR, R.hp * vgL));
}

// the other volume fluxes: sum_n g_n f#_n with the Cartesian direction fluxes
// (s0 = rho, s1 = p)
template <int VF>
__device__ __forceinline__ void generic_contra(const CPrim& L, const CPrim& R, const double g[3],
                                               double gm1inv, double f[5]) {
  Prim<double, 3> a, b;
  a.rho = L.s0;
  a.p = L.s1;
  b.rho = R.s0;
  b.p = R.s1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    a.v[k] = L.v[k];
    b.v[k] = R.v[k];
  }
  double f0[5], f1[5], f2[5];
  volume_flux<VF, double, 3, 0>(a, b, gm1inv, f0);
  volume_flux<VF, double, 3, 1>(a, b, gm1inv, f1);
  volume_flux<VF, double, 3, 2>(a, b, gm1inv, f2);
#pragma unroll
  for (int v = 0; v < 5; ++v) f[v] = fma(g[2], f2[v], fma(g[1], f1[v], g[0] * f0[v]));
}

// ---- surface flux along the metric vector g (length |g|) ----
__device__ __forceinline__ void contra_phys(const double* c, const Prim<double, 3>& q,
                                            const double g[3], double& vg, double f[5]) {
  vg = fma(q.v[2], g[2], fma(q.v[1], g[1], q.v[0] * g[0]));
  f[0] = fma(c[3], g[2], fma(c[2], g[1], c[1] * g[0]));
#pragma unroll
  for (int k = 0; k < 3; ++k) f[1 + k] = fma(c[1 + k], vg, q.p * g[k]);
  f[4] = (c[4] + q.p) * vg;
}

__device__ __forceinline__ void curved_surface_flux(int sf, const double* cl, const double* cr,
                                                    const double g[3], double gamma, double gm1,
                                                    double f[5]) {
  double rrl, rrr;
  const Prim<double, 3> ql = prim_rcp<3>(cl, gm1, rrl);
  const Prim<double, 3> qr = prim_rcp<3>(cr, gm1, rrr);
  if (sf == kSRanocha || sf == kSChandrashekar) {
    CPrim L, R;
    if (sf == kSRanocha) {
      L.s0 = 0.5 * ql.rho;
      L.s1 = gm1 * ql.rho * rcp(ql.p);
      R.s0 = 0.5 * qr.rho;
      R.s1 = gm1 * qr.rho * rcp(qr.p);
    } else {
      L.s0 = ql.rho;
      L.s1 = ql.p;
      R.s0 = qr.rho;
      R.s1 = qr.p;
    }
    L.hp = 0.5 * ql.p;
    R.hp = 0.5 * qr.p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      L.v[k] = ql.v[k];
      L.hv[k] = 0.5 * ql.v[k];
      R.v[k] = qr.v[k];
      R.hv[k] = 0.5 * qr.v[k];
    }
    if (sf == kSRanocha) ranocha_contra(L, R, g, f);
    else generic_contra<kVChandrashekar>(L, R, g, 1.0 / gm1, f);
    return;
  }
  double fl[5], fr[5], vgl, vgr;
  contra_phys(cl, ql, g, vgl, fl);
  contra_phys(cr, qr, g, vgr, fr);
  const double gn = sqrt(fma(g[2], g[2], fma(g[1], g[1], g[0] * g[0])));
  const double c2l = gamma * ql.p * rrl, c2r = gamma * qr.p * rrr;
  if (sf == kSLLF) {
    // lambda |g| = max(|v_L . g|, |v_R . g|) + max(c_L, c_R) |g|
    const double lam = fmax(fabs(vgl), fabs(vgr)) + sqrt(fmax(c2l, c2r)) * gn;
#pragma unroll
    for (int v = 0; v < 5; ++v) f[v] = 0.5 * (fl[v] + fr[v]) - 0.5 * lam * (cr[v] - cl[v]);
    return;
  }
  // HLL with Davis signal speeds along g (all speeds scaled by |g|)
  const double cgl = sqrt(c2l) * gn, cgr = sqrt(c2r) * gn;
  const double sL = fmin(vgl - cgl, vgr - cgr), sR = fmax(vgl + cgl, vgr + cgr);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    if (sL >= 0.0) f[v] = fl[v];
    else if (sR <= 0.0) f[v] = fr[v];
    else f[v] = (sR * fl[v] - sL * fr[v] + sL * sR * (cr[v] - cl[v])) / (sR - sL);
  }
}

// face-parallel: blockIdx.y = reference direction r; fs[r][v][e_left][l]
template <int N>
__global__ void curved_surface_kernel(const double* __restrict__ u, double* __restrict__ fs,
                                      const double* __restrict__ Ja, Geom g, int sf) {
  constexpr int NP = N + 1, P = NP * NP * NP, NF = NP * NP, NV = 5;
  const int r = blockIdx.y;
  const long long total = g.nelem * NF;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t / NF), l = (int)(t % NF);
    const int er = neighbour32(g, e, r, +1);
    const int nl = line_node_rt<3, N>(r, l, N), nr = line_node_rt<3, N>(r, l, 0);
    double cl[NV], cr[NV], gv[3];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      cl[v] = u[((long long)e * NV + v) * P + nl];
      cr[v] = u[((long long)er * NV + v) * P + nr];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) gv[k] = Ja[(((long long)e * 3 + r) * 3 + k) * P + nl];
    double f[NV];
    curved_surface_flux(sf, cl, cr, gv, g.gamma, g.gm1, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) fs[((long long)r * NV + v) * total + t] = f[v];
  }
}

// ---- volume: flux differencing, lifting, 1/J, source, optional stage update ----
template <int N>
struct CLaunch {
  static constexpr int NP = N + 1, P = NP * NP * NP, LINES = NP * NP;
  static constexpr int NC = 9;  // s0, s1, p/2, v[3], v[3]/2
  static constexpr int PER_ELEM = (NC + 3 + 5) * P * (int)sizeof(double);
  static constexpr int BY_THREADS = (128 / LINES) > 0 ? (128 / LINES) : 1;
  static constexpr int BY_SMEM = (98304 / PER_ELEM) > 0 ? (98304 / PER_ELEM) : 1;
  static constexpr int EPB = BY_THREADS < BY_SMEM ? BY_THREADS : BY_SMEM;
  static constexpr int SMEM = EPB * PER_ELEM;
};

template <int N, int VF, int EPB>
__device__ __forceinline__ void curved_direction(int r, double (*sp)[9][(N + 1) * (N + 1) * (N + 1)],
                                                 double (*sg)[3][(N + 1) * (N + 1) * (N + 1)],
                                                 double (*sa)[5][(N + 1) * (N + 1) * (N + 1)],
                                                 int el, int l, const CTables& tb, double gm1inv,
                                                 const double* __restrict__ fs, int nelem, int e,
                                                 int eleft) {
  constexpr int NP = N + 1, NV = 5, LINES = NP * NP;
  int node[NP];
  CPrim q[NP];
  double hg[NP][3];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    node[a] = line_node_rt<3, N>(r, l, a);
    const int nd = node[a];
    q[a].s0 = sp[el][0][nd];
    q[a].s1 = sp[el][1][nd];
    q[a].hp = sp[el][2][nd];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      q[a].v[k] = sp[el][3 + k][nd];
      q[a].hv[k] = sp[el][6 + k][nd];
      hg[a][k] = sg[el][k][nd];
    }
  }
  // the line sums continue the running totals of the earlier directions
  double acc[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[a][v] = sa[el][v][node[a]];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = a + 1; b < NP; ++b) {
      double gv[3], f[NV];
#pragma unroll
      for (int k = 0; k < 3; ++k) gv[k] = hg[a][k] + hg[b][k];
      if (VF == kVRanocha) ranocha_contra(q[a], q[b], gv, f);
      else generic_contra<VF>(q[a], q[b], gv, gm1inv, f);
      const double dab = tb.Ds[a][b], dba = tb.Ds[b][a];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[a][v] = fma(dab, f[v], acc[a][v]);
        acc[b][v] = fma(dba, f[v], acc[b][v]);
      }
    }
  }
  // lifting: this element's right face (its own flux) at node N, the left
  // neighbour's face at node 0; l indexes the face node
  const long long base = (long long)nelem * LINES;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const long long row = (long long)(r * NV + v) * base;
    acc[N][v] = fma(tb.liftR, fs[row + (long long)e * LINES + l], acc[N][v]);
    acc[0][v] = fma(tb.liftL, fs[row + (long long)eleft * LINES + l], acc[0][v]);
  }
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) sa[el][v][node[a]] = acc[a][v];
}

// N = 3: three CTAs per SM (168 registers, the shared memory of three
// 8-element CTAs fits the maximum carveout)
template <int N, int VF, int EPB>
__global__ void __launch_bounds__(EPB*(N + 1) * (N + 1), (N == 3 && EPB == 8) ? 3 : 1)
    curved_volume_kernel(double* u, double* __restrict__ du, const double* __restrict__ fs,
                         const double* __restrict__ Ja, const double* __restrict__ invJ,
                         const double* __restrict__ X, Geom g, CTables tb,
                         unsigned* __restrict__ err, StageFuse fz, SourceArgs src) {
  constexpr int NP = N + 1, P = NP * NP * NP, NV = 5, LINES = NP * NP, NC = 9;
  extern __shared__ __align__(16) unsigned char dg_smem[];
  double(*sp)[NC][P] = reinterpret_cast<double(*)[NC][P]>(dg_smem);
  double(*sg)[3][P] = reinterpret_cast<double(*)[3][P]>(dg_smem + sizeof(double) * EPB * NC * P);
  double(*sa)[NV][P] =
      reinterpret_cast<double(*)[NV][P]>(dg_smem + sizeof(double) * EPB * (NC + 3) * P);
  __shared__ int s_left[EPB][3];
  const int e0 = blockIdx.x * EPB;
  const int nelem = (int)g.nelem;
  if (threadIdx.x < EPB && e0 + (int)threadIdx.x < nelem) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
      s_left[threadIdx.x][r] = neighbour32(g, e0 + (int)threadIdx.x, r, -1);
  }
  unsigned bad = 0;
  for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
    const int el = t / P, node = t % P, e = e0 + el;
    if (e >= nelem) continue;
    double c[NV], rr;
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = u[((long long)e * NV + v) * P + node];
    const Prim<double, 3> q = prim_rcp<3>(c, g.gm1, rr);
    bad |= prim_check(q);
    node_slots<VF, double>(q.rho, q.p, g.gm1, sp[el][0][node], sp[el][1][node]);
    sp[el][2][node] = 0.5 * q.p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sp[el][3 + k][node] = q.v[k];
      sp[el][6 + k][node] = 0.5 * q.v[k];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) sa[el][v][node] = 0.0;
  }
  if (bad) atomicOr(err, bad);
  const int el = threadIdx.x / LINES, l = threadIdx.x % LINES;
  const bool active = (e0 + el) < nelem;
#pragma unroll 1
  for (int r = 0; r < 3; ++r) {
    // this direction's metric vectors, halved (the pair average is a sum)
    for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
      const int ell = t / P, node = t % P, e = e0 + ell;
      if (e >= nelem) continue;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        sg[ell][k][node] = 0.5 * Ja[(((long long)e * 3 + r) * 3 + k) * P + node];
    }
    __syncthreads();
    if (active)
      curved_direction<N, VF, EPB>(r, sp, sg, sa, el, l, tb, g.gm1inv, fs, nelem, e0 + el,
                                   s_left[el][r]);
    __syncthreads();
  }
  const double dtv = fz.k ? *fz.dt : 0.0;
  double* const uo = fz.u_out ? fz.u_out : u;
  const double ts = src.kind ? source_time(src) : 0.0;
  for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
    const int ell = t / P, node = t % P, e = e0 + ell;
    if (e >= nelem) continue;
    const double ij = invJ[(long long)e * P + node];
    double S[NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (src.kind == kSourceManufactured)
      manufactured_source(X[((long long)e * 3 + 0) * P + node], X[((long long)e * 3 + 1) * P + node],
                          X[((long long)e * 3 + 2) * P + node], ts, g.gm1, S);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double val = fma(ij, sa[ell][v][node], S[v]);
      const long long i = ((long long)e * NV + v) * P + node;
      if (fz.k) {
        double kk = dtv * val;
        if (fz.a != 0.0) kk = fma(fz.a, fz.k[i], kk);
        fz.k[i] = kk;
        uo[i] = u[i] + fz.b * kk;
      } else {
        du[i] = val;
      }
    }
  }
}

// ---- volume, pair-parallel variant for small meshes ----
// One element per CTA; per direction, one thread per (line, node pair)
// evaluates the contravariant flux into shared memory, then one thread per
// node sums its line's pairs in ascending partner order and adds the
// lifting: the order of the line-owning kernel above, with the pair work
// spread over LINES * N (N+1) / 2 threads instead of LINES (a tiny mesh does
// not fill the GPU, and each thread's FP64 chain is its latency).
template <int N>
struct CPairs {
  static constexpr int NP = N + 1, P = NP * NP * NP, LINES = NP * NP;
  static constexpr int NPAIRS = N * (N + 1) / 2;
  static constexpr int WORK = LINES * NPAIRS;
  static constexpr int THREADS = WORK < 512 ? ((WORK + 31) / 32) * 32 : 512;
  static constexpr int SMEM = (9 + 3 + 5) * P * (int)sizeof(double) + WORK * 5 * (int)sizeof(double);
};

// pair (a, b), a < b, of index p in the order (0,1), (0,2), ..., (0,N), (1,2), ...
template <int N>
__device__ __forceinline__ void pair_of(int p, int& a, int& b) {
  a = 0;
  while (p >= N - a) {
    p -= N - a;
    ++a;
  }
  b = a + 1 + p;
}
template <int N>
__device__ __forceinline__ int pair_index(int a, int b) {  // a < b
  return a * N - a * (a - 1) / 2 + (b - a - 1);
}

// line l and position i along direction r of a node (inverse of line_node)
template <int N>
__device__ __forceinline__ void line_of(int r, int node, int& l, int& i) {
  constexpr int NP = N + 1;
  if (r == 0) {
    l = node / NP;
    i = node % NP;
  } else if (r == 1) {
    i = (node / NP) % NP;
    l = node % NP + NP * (node / (NP * NP));
  } else {
    i = node / (NP * NP);
    l = node % (NP * NP);
  }
}

template <int N, int VF>
__global__ void __launch_bounds__(CPairs<N>::THREADS)
    curved_volume_pp_kernel(double* u, double* __restrict__ du, const double* __restrict__ fs,
                            const double* __restrict__ Ja, const double* __restrict__ invJ,
                            const double* __restrict__ X, Geom g, CTables tb,
                            unsigned* __restrict__ err, StageFuse fz, SourceArgs src) {
  using C = CPairs<N>;
  constexpr int NP = C::NP, P = C::P, NV = 5, LINES = C::LINES, NPAIRS = C::NPAIRS;
  extern __shared__ __align__(16) unsigned char dg_smem[];
  double(*sp)[P] = reinterpret_cast<double(*)[P]>(dg_smem);                         // [9][P]
  double(*sg)[P] = reinterpret_cast<double(*)[P]>(dg_smem + sizeof(double) * 9 * P);  // [3][P]
  double(*sa)[P] = reinterpret_cast<double(*)[P]>(dg_smem + sizeof(double) * 12 * P); // [5][P]
  double* sf = reinterpret_cast<double*>(dg_smem + sizeof(double) * 17 * P);          // [WORK][5]
  const int e = blockIdx.x;
  __shared__ int s_left[3];
  if (threadIdx.x < 3) s_left[threadIdx.x] = neighbour32(g, e, threadIdx.x, -1);
  unsigned bad = 0;
  for (int node = threadIdx.x; node < P; node += blockDim.x) {
    double c[NV], rr;
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = u[((long long)e * NV + v) * P + node];
    const Prim<double, 3> q = prim_rcp<3>(c, g.gm1, rr);
    bad |= prim_check(q);
    node_slots<VF, double>(q.rho, q.p, g.gm1, sp[0][node], sp[1][node]);
    sp[2][node] = 0.5 * q.p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sp[3 + k][node] = q.v[k];
      sp[6 + k][node] = 0.5 * q.v[k];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) sa[v][node] = 0.0;
  }
  if (bad) atomicOr(err, bad);
  const long long base = (long long)g.nelem * LINES;
#pragma unroll 1
  for (int r = 0; r < 3; ++r) {
    for (int node = threadIdx.x; node < P; node += blockDim.x) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
        sg[k][node] = 0.5 * Ja[(((long long)e * 3 + r) * 3 + k) * P + node];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < C::WORK; w += blockDim.x) {
      const int l = w / NPAIRS;
      int a, b;
      pair_of<N>(w % NPAIRS, a, b);
      const int na = line_node_rt<3, N>(r, l, a), nb = line_node_rt<3, N>(r, l, b);
      CPrim qa, qb;
      double gv[3], f[NV];
      qa.s0 = sp[0][na];
      qa.s1 = sp[1][na];
      qa.hp = sp[2][na];
      qb.s0 = sp[0][nb];
      qb.s1 = sp[1][nb];
      qb.hp = sp[2][nb];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        qa.v[k] = sp[3 + k][na];
        qa.hv[k] = sp[6 + k][na];
        qb.v[k] = sp[3 + k][nb];
        qb.hv[k] = sp[6 + k][nb];
        gv[k] = sg[k][na] + sg[k][nb];
      }
      if (VF == kVRanocha) ranocha_contra(qa, qb, gv, f);
      else generic_contra<VF>(qa, qb, gv, g.gm1inv, f);
#pragma unroll
      for (int v = 0; v < NV; ++v) sf[w * NV + v] = f[v];
    }
    __syncthreads();
    for (int node = threadIdx.x; node < P; node += blockDim.x) {
      int l, i;
      line_of<N>(r, node, l, i);
      // continuing the running total, in the line-owning kernel's order
      double acc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] = sa[v][node];
      for (int j = 0; j < NP; ++j) {
        if (j == i) continue;
        const int p = j < i ? pair_index<N>(j, i) : pair_index<N>(i, j);
        const double dij = tb.Ds[i][j];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = fma(dij, sf[(l * NPAIRS + p) * NV + v], acc[v]);
      }
      if (i == N) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
          acc[v] = fma(tb.liftR, fs[(long long)(r * NV + v) * base + (long long)e * LINES + l], acc[v]);
      }
      if (i == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
          acc[v] = fma(tb.liftL, fs[(long long)(r * NV + v) * base + (long long)s_left[r] * LINES + l],
                       acc[v]);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) sa[v][node] = acc[v];
    }
    __syncthreads();
  }
  const double dtv = fz.k ? *fz.dt : 0.0;
  double* const uo = fz.u_out ? fz.u_out : u;
  const double ts = src.kind ? source_time(src) : 0.0;
  for (int node = threadIdx.x; node < P; node += blockDim.x) {
    const double ij = invJ[(long long)e * P + node];
    double S[NV] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (src.kind == kSourceManufactured)
      manufactured_source(X[((long long)e * 3 + 0) * P + node], X[((long long)e * 3 + 1) * P + node],
                          X[((long long)e * 3 + 2) * P + node], ts, g.gm1, S);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double val = fma(ij, sa[v][node], S[v]);
      const long long idx = ((long long)e * NV + v) * P + node;
      if (fz.k) {
        double kk = dtv * val;
        if (fz.a != 0.0) kk = fma(fz.a, fz.k[idx], kk);
        fz.k[idx] = kk;
        uo[idx] = u[idx] + fz.b * kk;
      } else {
        du[idx] = val;
      }
    }
  }
}

// ---- wave speeds for the CFL step: per element sum_r max_nodes
// (|v . J a^r| + c |J a^r|) / J, max over elements (ordered bits) ----
template <int N>
__global__ void curved_speed_kernel(const double* __restrict__ u, const double* __restrict__ Ja,
                                    const double* __restrict__ invJ, Geom g,
                                    unsigned long long* out, unsigned* err,
                                    double* __restrict__ copy_to) {
  constexpr int NP = N + 1, P = NP * NP * NP, NV = 5;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double best = 0.0;
  unsigned bad = 0;
  for (long long e = warp; e < g.nelem; e += nwarps) {
    double lam[3] = {0.0, 0.0, 0.0};
    for (int node = lane; node < P; node += 32) {
      double c[NV], rr;
#pragma unroll
      for (int v = 0; v < NV; ++v) c[v] = u[(e * NV + v) * P + node];
      if (copy_to) {
#pragma unroll
        for (int v = 0; v < NV; ++v) copy_to[(e * NV + v) * P + node] = c[v];
      }
      const Prim<double, 3> q = prim_rcp<3>(c, g.gm1, rr);
      bad |= prim_check(q);
      const double cs = sqrt(g.gamma * q.p * rr), ij = invJ[e * P + node];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double gv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) gv[k] = Ja[((e * 3 + r) * 3 + k) * P + node];
        const double vg = fma(q.v[2], gv[2], fma(q.v[1], gv[1], q.v[0] * gv[0]));
        const double gn = sqrt(fma(gv[2], gv[2], fma(gv[1], gv[1], gv[0] * gv[0])));
        lam[r] = fmax(lam[r], (fabs(vg) + cs * gn) * ij);
      }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
      for (int off = 16; off > 0; off >>= 1)
        lam[r] = fmax(lam[r], __shfl_xor_sync(0xffffffffu, lam[r], off));
    best = fmax(best, lam[0] + lam[1] + lam[2]);
  }
  __shared__ double sb[32];
  if (lane == 0) sb[threadIdx.x >> 5] = best;
  if (bad) atomicOr(err, bad);
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sb[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
  }
}

}  // namespace dg
