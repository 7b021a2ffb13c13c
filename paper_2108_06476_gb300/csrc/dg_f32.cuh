// FP32 arithmetic of the rhs in perturbation form (the precision pattern:
// FP32 volume and surface kernels, the state, the Runge-Kutta update and
// the reductions in FP64, and the logarithmic mean's small-difference branch
// in FP64).
//
// Why a perturbation form. The split-form rhs sums terms of size
// (2/h)|Dt||f| that cancel to |du|. On smooth flows the energy flux carries a
// large constant part, v_n p gamma/(gamma-1) (about 20 at p = 20, |v| = 0.3),
// while du_E is set by the kinetic energy's variation (about 0.1): a plain
// FP32 evaluation rounds the constant part at 6e-8 relative and loses 3 to 5
// of the 7 digits. Every row of the split-form operator annihilates a
// constant flux together with the lifting (sum_b Ds_ab + liftR [a = N] +
// liftL [a = 0] = 0, since Dt's rows sum to -(W^-1 B)_aa), so each element
// may subtract the flux of a reference state c_e = f(u_ref) from every
// two-point and surface flux it uses without changing du. This file
// evaluates f#(u_L, u_R) - f(u_ref) directly from the nodes' deviations
// (delta rho, delta v, delta p) from an FP32 reference (rho0, v0, p0) of the
// element, with the constant parts cancelled algebraically; the rounding is
// then relative to the variation inside the element, not to the state.
//
// The deviations are formed in FP64 from the FP64 state: delta rho = rho -
// rho0, delta m = m - rho v0 (so delta v = delta m / rho), delta E = E - E0
// with E0 = p0/(gamma-1) + rho0 |v0|^2/2, and then
//   delta p = (gamma-1) (delta E - (delta rho |v|^2 + rho0 delta v . (v + v0))/2).
//
// Ranocha's flux (ranocha2020icosahom) and Chandrashekar's flux share their
// mass flux f1 = ln_mean(rho) avg(v_n) and their internal-energy term
// avg(v_n) P / (gamma-1), P = ln_mean(rho) / ln_mean(rho/p) (the energy term
// of Ranocha's flux is f1 / ((gamma-1) ln_mean(rho/p)); Chandrashekar's
// f1 / (2 (gamma-1) ln_mean(beta)) with beta = rho/(2p) is the same). With
// s = x + y, t = (y - x)/s and ln_mean(x, y) = (s/2) Q(t^2), Q(t^2) =
// t / atanh(t):
//   P = H Q(a) / Q(b),  H = (rho_L + rho_R) / (rho_L/p_L + rho_R/p_R),
//   a = t_rho^2, b = t_sig^2 (t of rho and of sig = rho/p),
//   H - p0 = (rho_L p_R dp_L + rho_R p_L dp_R) / (rho_L p_R + rho_R p_L),
//   t_rho - t_sig = 2 rho_L rho_R (p_R - p_L) / ((rho_L + rho_R)(rho_R p_L + rho_L p_R)),
// and with phi = 1 - Q = f2 R(f2) the ratio is Q(a)/Q(b) - 1 =
// -(phi(a) - phi(b)) / Q(b), phi(a) - phi(b) = (a - b) [phi](a, b), the
// divided difference of a polynomial evaluated by a double Horner scheme:
// every quantity that vanishes for constant pressure vanishes exactly here,
// and small ones keep their relative accuracy. Chandrashekar's momentum
// pressure ({rho}/(2 {beta})) is H itself.
#pragma once
#include "dg_device.cuh"

namespace dg {

// ---- the log-mean polynomials of the perturbation form ----
// phi(f2) = 1 - t/atanh(t) = f2 R(f2). FP64 small-difference branch (both
// log means' f2 below kSeriesLim): the Taylor series of R to first order,
// evaluated in FP64; its truncation (the f2^2 term, 1.4e-9 relative at the
// limit) lies 40 times below the FP32 rounding of every result it feeds, and
// R(0) = 1/3 is exact. FP32 range f2 < 0.25: a fitted degree-5 R
// (gen_log_mean_poly.py); beyond, log1p. phi_r64 and phi_r32 state the
// polynomials; phi_r64_dd and phi_r32_dd evaluate the same coefficients.
constexpr float kSeriesLim = 1.0e-4f;
// degree 1 on f2 in [0, 1e-4]; measured relative error 1.4e-09
__device__ __forceinline__ double phi_r64(double f2) {
  double r = 0.08888888888888889;
  return fma(f2, r, 0.3333333333333333);
}
// degree 5 on f2 in [0, 0.25]; measured relative error 4.9e-08
__device__ __forceinline__ float phi_r32(float f2) {
  float r = 0.03261576220393181f;
  r = fmaf(f2, r, 0.0167341660708189f);
  r = fmaf(f2, r, 0.030890846624970436f);
  r = fmaf(f2, r, 0.046518709510564804f);
  r = fmaf(f2, r, 0.08888980746269226f);
  return fmaf(f2, r, 0.3333333432674408f);
}

// R(a) and the divided difference [R](a, b) = (R(a) - R(b))/(a - b) of the
// same polynomials: Horner's scheme at a keeps its partial sums s_k, and
// [R](a, b) is Horner's scheme at b over s_1..s_K (for the first-order
// series, the constant s_1).
__device__ __forceinline__ void phi_r64_dd(double a, double, double& Ra, double& dd) {
  const double s1 = 0.08888888888888889;
  Ra = fma(s1, a, 0.3333333333333333);
  dd = s1;
}
__device__ __forceinline__ void phi_r32_dd(float a, float b, float& Ra, float& dd) {
  const float s5 = 0.03261576220393181f;
  const float s4 = fmaf(s5, a, 0.0167341660708189f);
  const float s3 = fmaf(s4, a, 0.030890846624970436f);
  const float s2 = fmaf(s3, a, 0.046518709510564804f);
  const float s1 = fmaf(s2, a, 0.08888980746269226f);
  Ra = fmaf(s1, a, 0.3333333432674408f);
  dd = fmaf(fmaf(fmaf(fmaf(s5, b, s4), b, s3), b, s2), b, s1);
}

// Q(t^2) = t/atanh(t) for any |t| < 1 (far branch)
static __device__ __noinline__ float q_any32(float t) {
  const float f2 = t * t;
  if (f2 < 0.25f) return fmaf(-f2, phi_r32(f2), 1.0f);
  return 2.0f * t / log1pf(2.0f * t / (1.0f - t));
}

// element reference in normal-first order for one direction
template <int D>
struct DRef {
  float rho0, p0, K0, m0n;  // K0 = |v0|^2/2, m0n = rho0 v0_n
  float v0[D];
};

// node deviations (v, dv in natural order in shared memory; normal-first in
// a line)
template <int D>
struct DNode {
  float rho, drho, dp;
  float v[D], dv[D];
};

// FP64 state of one node -> FP32 deviations from the reference (rho0, v0,
// p0; E0 = p0/(gamma-1) + rho0 |v0|^2/2 in FP64), natural variable order.
// dm (optional) receives m - rho v0 and dEo E - E0 (the face kernels form
// the jumps of the conserved variables from them).
template <int D>
__device__ __forceinline__ void delta_node(const double* c, float rho0, const float* v0, double E0,
                                           float gm1f, DNode<D>& q, float* dm = nullptr,
                                           float* dEo = nullptr) {
  q.drho = d2f(c[0] - f2d(rho0));
  q.rho = rho0 + q.drho;
  const float rr = rcp(q.rho);
  float v2 = 0.0f, dvv = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float dmk = d2f(fma(-c[0], f2d(v0[k]), c[1 + k]));  // m - rho v0
    if (dm) dm[k] = dmk;
    q.dv[k] = dmk * rr;
    q.v[k] = v0[k] + q.dv[k];
    v2 = fmaf(q.v[k], q.v[k], v2);
    dvv = fmaf(q.dv[k], q.v[k] + v0[k], dvv);
  }
  const float dE = d2f(c[D + 1] - E0);
  if (dEo) *dEo = dE;
  q.dp = gm1f * fmaf(-0.5f, fmaf(q.drho, v2, rho0 * dvv), dE);
}

template <int D>
__device__ __forceinline__ double ref_energy(float rho0, const float* v0, float p0, double gm1inv) {
  double v2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) v2 = fma((double)v0[k], (double)v0[k], v2);
  return fma((double)p0, gm1inv, 0.5 * (double)rho0 * v2);
}

struct DLogMeans {
  float drl;  // ln_mean(rho_L, rho_R) - rho0
  float dH;   // H - p0
  float dPh;  // P - p0, P = ln_mean(rho) / ln_mean(rho/p)
};

__device__ __forceinline__ DLogMeans delta_log_means(float rL, float rR, float drL, float drR,
                                                     float pL, float pR, float dpL, float dpR,
                                                     float p0) {
  const float S = rL + rR;
  const float iS = rcp(S);
  const float t = (drR - drL) * iS;
  const float W = fmaf(rL, pR, rR * pL);
  const float iW = rcp(W);
  const float dH = fmaf(rL * pR, dpL, (rR * pL) * dpR) * iW;
  const float Dt = ((2.0f * rL) * rR) * (dpR - dpL) * (iS * iW);
  const float ts = t - Dt;  // t of sig = rho/p
  const float dts = t - ts;  // exact for small differences (Sterbenz)
  float phia, r;
  const float a = t * t, b = ts * ts;
  if (fmaxf(a, b) < kSeriesLim) {
    // small-difference branch: the series of R and its divided difference
    // in FP64
    double Ra, dd;
    const double bd = f2d(b);
    phi_r64_dd(f2d(a), bd, Ra, dd);
    const float dphi = (dts * (t + ts)) * d2f(fma(bd, dd, Ra));  // phi(a) - phi(b)
    phia = a * d2f(Ra);
    r = -dphi * rcp(1.0f - phia + dphi);
  } else if (fmaxf(a, b) < 0.25f) {
    // FP32 polynomial range
    float Ra, dd;
    phi_r32_dd(a, b, Ra, dd);
    const float dphi = (dts * (t + ts)) * fmaf(b, dd, Ra);
    phia = a * Ra;
    r = -dphi * rcp(1.0f - phia + dphi);
  } else {
    // far from x = y
    const float qa = q_any32(t), qb = q_any32(ts);
    phia = 1.0f - qa;
    r = (qa - qb) * rcp(qb);  // exactly 0 when t_sig = t_rho (constant pressure)
  }
  DLogMeans o;
  o.drl = fmaf(-0.5f * S, phia, 0.5f * (drL + drR));
  o.dH = dH;
  o.dPh = fmaf(p0 + dH, r, dH);
  return o;
}

// f#(L, R) - f(ref) for Ranocha's (VF = kVRanocha) or Chandrashekar's flux,
// normal-first order
template <int VF, int D>
__device__ __forceinline__ void delta_pair(const DNode<D>& L, const DNode<D>& R, const DRef<D>& rf,
                                           float gm1inv, float f[D + 2]) {
  const float pL = rf.p0 + L.dp, pR = rf.p0 + R.dp;
  const DLogMeans lm = delta_log_means(L.rho, R.rho, L.drho, R.drho, pL, pR, L.dp, R.dp, rf.p0);
  float vb[D], dvb[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    vb[k] = 0.5f * (L.v[k] + R.v[k]);
    dvb[k] = 0.5f * (L.dv[k] + R.dv[k]);
  }
  const float dpb = 0.5f * (L.dp + R.dp);
  const float df1 = fmaf(lm.drl, vb[0], rf.rho0 * dvb[0]);
  f[0] = df1;
#pragma unroll
  for (int k = 0; k < D; ++k) f[1 + k] = fmaf(df1, vb[k], rf.m0n * dvb[k]);
  f[1] += (VF == kVRanocha) ? dpb : lm.dH;
  // v_L.v_R/2 - |v0|^2/2 = v0 . dv_avg + dv_L . dv_R / 2
  float dll = 0.0f, v0d = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    dll = fmaf(L.dv[k], R.dv[k], dll);
    v0d = fmaf(rf.v0[k], dvb[k], v0d);
  }
  const float dK = fmaf(0.5f, dll, v0d);
  const float Ph = rf.p0 + lm.dPh;
  float fe = fmaf(df1, rf.K0 + dK, rf.m0n * dK);
  fe = fmaf(fmaf(dvb[0], Ph, rf.v0[0] * lm.dPh), gm1inv, fe);
  if (VF == kVRanocha)
    fe += fmaf(rf.p0, dvb[0], fmaf(rf.v0[0], dpb, 0.5f * fmaf(L.dp, R.dv[0], R.dp * L.dv[0])));
  else
    fe += fmaf(lm.dH, vb[0], rf.p0 * dvb[0]);
  f[D + 1] = fe;
}

// f(X) - f(ref) of the Euler flux, normal-first; ggm1 = gamma/(gamma-1)
template <int D>
__device__ __forceinline__ void delta_phys_flux(const DNode<D>& X, const DRef<D>& rf, float ggm1,
                                                float f[D + 2]) {
  const float dm = fmaf(X.drho, X.v[0], rf.rho0 * X.dv[0]);  // rho v_n - rho0 v0_n
  f[0] = dm;
#pragma unroll
  for (int k = 0; k < D; ++k) f[1 + k] = fmaf(dm, X.v[k], rf.m0n * X.dv[k]);
  f[1] += X.dp;
  float v2 = 0.0f, dvv = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v2 = fmaf(X.v[k], X.v[k], v2);
    dvv = fmaf(X.dv[k], X.v[k] + rf.v0[k], dvv);
  }
  // (E + p) v_n = rho |v|^2 v_n / 2 + gamma/(gamma-1) p v_n
  f[D + 1] = fmaf(0.5f, fmaf(dm, v2, rf.m0n * dvv), ggm1 * fmaf(X.dp, X.v[0], rf.p0 * X.dv[0]));
}

// reference flux f_dir(ref) in FP64 (natural variable order); ref values are
// FP32 numbers widened exactly
template <int D>
__device__ __forceinline__ void ref_flux64(const float* ref, int dir, double gamma, double gm1inv,
                                           double f[D + 2]) {
  const double rho0 = ref[0], p0 = ref[D + 1];
  double v2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) v2 = fma((double)ref[1 + k], (double)ref[1 + k], v2);
  const double vn = ref[1 + dir];
  const double m = rho0 * vn;
  f[0] = m;
#pragma unroll
  for (int k = 0; k < D; ++k) f[1 + k] = m * (double)ref[1 + k];
  f[1 + dir] += p0;
  f[D + 1] = vn * fma(p0 * gamma, gm1inv, 0.5 * rho0 * v2);
}

// per-element FP32 reference (rho0, v0, p0) from one node of the element:
// ref[e][0] = rho0, ref[e][1..D] = v0, ref[e][D+1] = p0, and its FP64 energy
// refE[e] = E0 = p0/(gamma-1) + rho0 |v0|^2/2. Any nearby state serves; the
// arithmetic of the perturbation form is exact in it.
// The reference is the state of the element's central node ((N/2, N/2[,
// N/2]) in node indices), which halves the largest deviation inside the
// element against a corner node.
template <int D>
__device__ __forceinline__ void element_ref(const double* __restrict__ u,
                                            float* __restrict__ ref, double* __restrict__ refE,
                                            long long e, int NP, double gm1, double gm1inv) {
  constexpr int NV = D + 2;
  const int P = (D == 2) ? NP * NP : NP * NP * NP;
  const int cn = (NP - 1) / 2;
  const int node = (D == 2) ? cn * (1 + NP) : cn * (1 + NP + NP * NP);
  const double* c = u + e * NV * P + node;
  const double rho = c[0];
  const double rr = 1.0 / rho;
  double mv = 0.0;
  float* o = ref + e * NV;
  float v0[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double m = c[(1 + k) * P];
    v0[k] = (float)(m * rr);
    o[1 + k] = v0[k];
    mv = fma(m, (double)v0[k], mv);
  }
  const float rho0 = (float)rho;
  const float p0 = (float)(gm1 * fma(-0.5, mv, c[(D + 1) * P]));
  o[0] = rho0;
  o[D + 1] = p0;
  refE[e] = ref_energy<D>(rho0, v0, p0, gm1inv);
}

template <int D>
__global__ void ref_kernel(const double* __restrict__ u, float* __restrict__ ref,
                           double* __restrict__ refE, long long nelem, int NP, double gm1,
                           double gm1inv) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nelem;
       e += (long long)gridDim.x * blockDim.x)
    element_ref<D>(u, ref, refE, e, NP, gm1, gm1inv);
}

template <int D>
__device__ __forceinline__ void load_ref(const float* __restrict__ ref, long long e, float& rho0,
                                         float* v0, float& p0) {
  const float* r = ref + e * (D + 2);
  rho0 = r[0];
#pragma unroll
  for (int k = 0; k < D; ++k) v0[k] = r[1 + k];
  p0 = r[D + 1];
}

// the reference of one direction, normal-first (t1 = dir+1, t2 = dir+2 mod D)
template <int D>
__device__ __forceinline__ DRef<D> dir_ref(float rho0, const float* v0, float p0, int dir) {
  DRef<D> r;
  r.rho0 = rho0;
  r.p0 = p0;
  float k0 = 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) k0 = fmaf(v0[k], v0[k], k0);
  r.K0 = 0.5f * k0;
  r.v0[0] = v0[dir];
  r.v0[1] = v0[(dir + 1) % D];
  if (D == 3) r.v0[D - 1] = v0[(dir + 2) % D];
  r.m0n = rho0 * r.v0[0];
  return r;
}

template <int D>
__device__ __forceinline__ DNode<D> to_normal_first(const DNode<D>& q, int dir) {
  DNode<D> o;
  o.rho = q.rho;
  o.drho = q.drho;
  o.dp = q.dp;
  const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  o.v[0] = q.v[dir];
  o.dv[0] = q.dv[dir];
  o.v[1] = q.v[t1];
  o.dv[1] = q.dv[t1];
  if (D == 3) {
    o.v[D - 1] = q.v[t2];
    o.dv[D - 1] = q.dv[t2];
  }
  return o;
}

// F*(u_L, u_R) - f(ref of the left element), normal-first. du[] holds
// fl32(u_R - u_L) (FP64 differences), normal-first; gamma, gm1inv, ggm1 in
// FP32.
template <int D>
__device__ __forceinline__ void delta_surface_flux(int sf, const DNode<D>& L, const DNode<D>& R,
                                                   const DRef<D>& rf, const float* du, float gamma,
                                                   float gm1inv, float ggm1, float f[D + 2]) {
  if (sf == kSRanocha) {
    delta_pair<kVRanocha, D>(L, R, rf, gm1inv, f);
    return;
  }
  if (sf == kSChandrashekar) {
    delta_pair<kVChandrashekar, D>(L, R, rf, gm1inv, f);
    return;
  }
  float fl[D + 2], fr[D + 2];
  delta_phys_flux<D>(L, rf, ggm1, fl);
  delta_phys_flux<D>(R, rf, ggm1, fr);
  const float pL = rf.p0 + L.dp, pR = rf.p0 + R.dp;
  const float c2l = gamma * pL * rcp(L.rho), c2r = gamma * pR * rcp(R.rho);
  if (sf == kSLLF) {
    const float lam = fmaxf(fabsf(L.v[0]), fabsf(R.v[0])) + sqrtf(fmaxf(c2l, c2r));
#pragma unroll
    for (int v = 0; v < D + 2; ++v) f[v] = 0.5f * ((fl[v] + fr[v]) - lam * du[v]);
    return;
  }
  const float cl = sqrtf(c2l), cr = sqrtf(c2r);
  const float sL = fminf(L.v[0] - cl, R.v[0] - cr);
  const float sR = fmaxf(L.v[0] + cl, R.v[0] + cr);
#pragma unroll
  for (int v = 0; v < D + 2; ++v) {
    if (sL >= 0.0f) f[v] = fl[v];
    else if (sR <= 0.0f) f[v] = fr[v];
    else f[v] = (sR * fl[v] - sL * fr[v] + sL * sR * du[v]) / (sR - sL);
  }
}

}  // namespace dg
