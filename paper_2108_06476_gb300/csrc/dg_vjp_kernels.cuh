// Vector-Jacobian product of the rhs: ubar = (d rhs / d u)^T w.
//
// The rhs is a sum of two-point terms. A volume pair (a, b) on a line in
// direction k contributes Ds[a][b] f#(u_a, u_b) to du_a and Ds[b][a] f#(u_a, u_b)
// to du_b, so its cotangent is g = Ds[a][b] w_a + Ds[b][a] w_b and it adds
// (d f#/d u_a)^T g to ubar_a and (d f#/d u_b)^T g to ubar_b. A face adds
// liftR F* to du at node N of its left element and liftL F* at node 0 of its
// right element: g = liftR w_L + liftL w_R, ubar_L += (dF*/du_L)^T g,
// ubar_R += (dF*/du_R)^T g. The flux Jacobians come from forward-mode dual
// numbers seeded with the 2 (d+2) conserved components of the two states; the
// two-point fluxes are recomputed, nothing is stored from the forward pass.
//
//  vjp_face_kernel: one thread per face node; writes the two adjoint
//    contributions of every face to fb[dir][side][v][e_left][l].
//  vjp_volume_kernel: one thread per element line, one direction at a time
//    (as the volume kernel), accumulating ubar in shared memory; the epilogue
//    adds the face contributions and stores ubar.
#pragma once
#include "dg_rhs_kernels.cuh"
#include "dg_dual.cuh"

namespace dg {

// physical index of normal-first component c in direction dir
template <int D>
__device__ __forceinline__ int nf_index(int dir, int c) {
  if (c == 0) return 0;
  if (c == D + 1) return D + 1;
  return 1 + (dir + c - 1) % D;
}

// adjoint of one two-point flux: ga = (df/du_a)^T g, gb = (df/du_b)^T g,
// everything in normal-first order (direction = component 1)
template <typename R, int D>
__device__ __forceinline__ void pair_vjp(int vf, int sf, bool surface, const R* ua, const R* ub,
                                         const R* g, R gamma, R gm1, R gm1inv, R* ga, R* gb) {
  constexpr int NV = D + 2, K = 2 * NV;
  using DT = Dual<R, K>;
  DT ca[NV], cb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    ca[v] = DT(ua[v]);
    ca[v].d[v] = R(1);
    cb[v] = DT(ub[v]);
    cb[v].d[NV + v] = R(1);
  }
  const Prim<DT, D> qa = cons2prim<DT, D>(ca, DT(gm1));
  const Prim<DT, D> qb = cons2prim<DT, D>(cb, DT(gm1));
  DT f[NV];
  if (surface) {
    surface_flux_dir<DT, D, 0>(sf, ca, cb, qa, qb, DT(gamma), DT(gm1inv), f);
  } else if (vf == kVRanocha) {
    flux_ranocha<DT, D, 0>(qa, qb, DT(gm1inv), f);
  } else if (vf == kVChandrashekar) {
    flux_chandrashekar<DT, D, 0>(qa, qb, DT(gm1inv), f);
  } else {
    flux_central<DT, D, 0>(qa, qb, DT(gm1inv), f);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    R sa = R(0), sb = R(0);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      sa = ::fma(g[k], f[k].d[v], sa);
      sb = ::fma(g[k], f[k].d[NV + v], sb);
    }
    ga[v] = sa;
    gb[v] = sb;
  }
}

// Reverse mode for Ranocha's volume flux, on primitive variables: the adjoint
// of one two-point flux f#(q_a, q_b) (q = (rho, v normal-first, p)) for the
// cotangent g (normal-first), added to ba and bb (adjoints of q_a, q_b). The
// flux is flux_ranocha's:
//   f_rho = L(rho_a, rho_b) vn,   vn = (v_a,n + v_b,n)/2,
//   f_m_k = f_rho (v_a,k + v_b,k)/2 + delta_kn (p_a + p_b)/2,
//   f_E   = f_rho (v_a . v_b / 2 + p_a p_b I / (gamma - 1)) + (p_a v_b,n + p_b v_a,n)/2,
//   I = 1/L(rho_a p_b, rho_b p_a),
// and its adjoint is written out term by term; only the two logarithmic means
// are differentiated forward, as functions of two arguments (dual numbers of
// two components).
template <typename R, int D>
__device__ __forceinline__ void ranocha_pair_rev(const R* qa, const R* qb, const R* g, R gm1inv,
                                                 R* ba, R* bb) {
  using D2 = Dual<R, 2>;
  const R ra = qa[0], rb = qb[0], pa = qa[D + 1], pb = qb[D + 1];
  D2 xa(ra), xb(rb);
  xa.d[0] = R(1);
  xb.d[1] = R(1);
  const D2 rl = ln_mean(xa, xb);
  D2 X(ra * pb), Y(rb * pa);
  X.d[0] = R(1);
  Y.d[1] = R(1);
  const D2 I = inv_ln_mean(X, Y);
  R vdot = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) vdot += qa[1 + k] * qb[1 + k];
  const R an = R(0.5) * (qa[1] + qb[1]);
  const R f0 = rl.v * an;
  const R eterm = R(0.5) * vdot + pa * pb * I.v * gm1inv;
  const R gE = g[D + 1];
  // the cotangent of f_rho, and the velocity terms of the momentum flux
  R f0b = g[0] + gE * eterm;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    f0b += g[1 + k] * (R(0.5) * (qa[1 + k] + qb[1 + k]));
    const R t = R(0.5) * g[1 + k] * f0;
    ba[1 + k] += t;
    bb[1 + k] += t;
  }
  // pressure average in the normal momentum
  ba[D + 1] += R(0.5) * g[1];
  bb[D + 1] += R(0.5) * g[1];
  // energy: v_a . v_b / 2, the pressure-velocity terms, p_a p_b I / (gamma - 1)
  const R vdb = R(0.5) * gE * f0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    ba[1 + k] += vdb * qb[1 + k];
    bb[1 + k] += vdb * qa[1 + k];
  }
  ba[D + 1] += R(0.5) * gE * qb[1];
  bb[1] += R(0.5) * gE * pa;
  bb[D + 1] += R(0.5) * gE * qa[1];
  ba[1] += R(0.5) * gE * pb;
  const R ipmb = gE * f0 * gm1inv;
  ba[D + 1] += ipmb * pb * I.v;
  bb[D + 1] += ipmb * pa * I.v;
  const R Ib = ipmb * pa * pb;
  const R Xb = Ib * I.d[0], Yb = Ib * I.d[1];
  ba[0] += Xb * pb;
  bb[D + 1] += Xb * ra;
  bb[0] += Yb * pa;
  ba[D + 1] += Yb * rb;
  // f_rho = L(rho_a, rho_b) vn
  const R rlb = f0b * an, anb = f0b * rl.v;
  ba[1] += R(0.5) * anb;
  bb[1] += R(0.5) * anb;
  ba[0] += rlb * rl.d[0];
  bb[0] += rlb * rl.d[1];
}

// Reverse mode for the LLF surface flux F* = (f(u_L) + f(u_R))/2 - lam (u_R -
// u_L)/2, lam = max(|v_n,L|, |v_n,R|) + max(c_L, c_R), in normal-first
// conserved variables: gl = J(u_L)^T g / 2 + lam g / 2 - (g . (u_R - u_L))
// dlam/du_L / 2 and gr likewise, with the Euler flux Jacobian's transpose
// written out (H = (E + p)/rho):
//   (J^T g)_rho = g_1 (gm1 |v|^2/2 - v_n^2) - sum_t g_t v_t v_n + g_E v_n (gm1 |v|^2/2 - H)
//   (J^T g)_mn  = g_0 + g_1 (2 - gm1) v_n + sum_t g_t v_t + g_E (H - gm1 v_n^2)
//   (J^T g)_mt  = -g_1 gm1 v_t + g_t v_n - g_E gm1 v_t v_n
//   (J^T g)_E   = g_1 gm1 + g_E gamma v_n
// and the derivative of lam taken along its maxima (ties: the left state;
// d|x|/dx = +1 at 0), as the dual-number evaluation of the same flux does.
template <typename R, int D>
__device__ __forceinline__ void llf_side_rev(const R* c, const R* g, R gamma, R gm1, R half_lam,
                                             R* out) {
  constexpr int NV = D + 2;
  const R rho = c[0], ir = R(1) / rho;
  R v[D], v2 = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v[k] = c[1 + k] * ir;
    v2 += v[k] * v[k];
  }
  const R p = gm1 * (c[NV - 1] - R(0.5) * rho * v2);
  const R H = (c[NV - 1] + p) * ir, vn = v[0], k2 = R(0.5) * gm1 * v2;
  R gtv = R(0), gtvs = R(0);  // sum_t g_t v_t
#pragma unroll
  for (int k = 1; k < D; ++k) gtv += g[1 + k] * v[k];
  gtvs = gtv;
  out[0] = R(0.5) * (g[1] * (k2 - vn * vn) - gtvs * vn + g[NV - 1] * vn * (k2 - H)) + half_lam * g[0];
  out[1] = R(0.5) * (g[0] + g[1] * (R(2) - gm1) * vn + gtv + g[NV - 1] * (H - gm1 * vn * vn)) +
           half_lam * g[1];
#pragma unroll
  for (int k = 1; k < D; ++k)
    out[1 + k] = R(0.5) * (-g[1] * gm1 * v[k] + g[1 + k] * vn - g[NV - 1] * gm1 * v[k] * vn) +
                 half_lam * g[1 + k];
  out[NV - 1] = R(0.5) * (g[1] * gm1 + g[NV - 1] * gamma * vn) + half_lam * g[NV - 1];
}

// d|v_n|/du and dc/du of one state (normal-first conserved), scaled by s
template <typename R, int D>
__device__ __forceinline__ void lam_terms(const R* c, R gamma, R gm1, bool take_v, bool take_c,
                                          R s, R* out) {
  constexpr int NV = D + 2;
  const R rho = c[0], ir = R(1) / rho;
  R v[D], v2 = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v[k] = c[1 + k] * ir;
    v2 += v[k] * v[k];
  }
  if (take_v) {
    const R sg = v[0] < R(0) ? R(-1) : R(1);
    out[0] += s * sg * (-v[0] * ir);
    out[1] += s * sg * ir;
  }
  if (take_c) {
    const R p = gm1 * (c[NV - 1] - R(0.5) * rho * v2);
    const R cs = ::sqrt(gamma * p * ir);
    const R a = gamma / (R(2) * cs * rho);
    out[0] += s * a * (gm1 * R(0.5) * v2 - p * ir);
#pragma unroll
    for (int k = 0; k < D; ++k) out[1 + k] += s * a * (-gm1 * v[k]);
    out[NV - 1] += s * a * gm1;
  }
}

template <typename R, int D>
__device__ __forceinline__ void llf_rev(const R* cl, const R* cr, const R* g, R gamma, R gm1,
                                        R* gl, R* gr) {
  constexpr int NV = D + 2;
  // lam from the two states, as the flux computes it
  const R irl = R(1) / cl[0], irr = R(1) / cr[0];
  R v2l = R(0), v2r = R(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    v2l += (cl[1 + k] * irl) * (cl[1 + k] * irl);
    v2r += (cr[1 + k] * irr) * (cr[1 + k] * irr);
  }
  const R vnl = cl[1] * irl, vnr = cr[1] * irr;
  const R pl = gm1 * (cl[NV - 1] - R(0.5) * cl[0] * v2l);
  const R pr = gm1 * (cr[NV - 1] - R(0.5) * cr[0] * v2r);
  const R csl = ::sqrt(gamma * pl * irl), csr = ::sqrt(gamma * pr * irr);
  const bool vleft = ::fabs(vnl) >= ::fabs(vnr), cleft = csl >= csr;
  const R lam = (vleft ? ::fabs(vnl) : ::fabs(vnr)) + (cleft ? csl : csr);
  llf_side_rev<R, D>(cl, g, gamma, gm1, R(0.5) * lam, gl);
  llf_side_rev<R, D>(cr, g, gamma, gm1, R(-0.5) * lam, gr);
  R jump = R(0);
#pragma unroll
  for (int v = 0; v < NV; ++v) jump += g[v] * (cr[v] - cl[v]);
  const R s = R(-0.5) * jump;
  lam_terms<R, D>(cl, gamma, gm1, vleft, cleft, s, gl);
  lam_terms<R, D>(cr, gamma, gm1, !vleft, !cleft, s, gr);
}

template <int D, int N, typename R, int dir>
__device__ __forceinline__ void vjp_face_body(const double* __restrict__ u,
                                              const double* __restrict__ w,
                                              double* __restrict__ fb, const Geom& g,
                                              const Tables<double>& tb, int sf) {
  using S = Shape<D, N>;
  constexpr int NV = S::NV, P = S::P, NF = S::LINES;
  const int nelem = (int)g.nelem;
  const long long total = (long long)nelem * NF;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t / NF), l = (int)(t % NF);
    const int er = neighbour32(g, e, dir, +1);
    const int nl = line_node<D, N, dir>(l, N), nr = line_node<D, N, dir>(l, 0);
    R ul[NV], ur[NV], gg[NV], gl[NV], gr[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const int v = nf_index<D>(dir, c);
      ul[c] = R(u[((long long)e * NV + v) * P + nl]);
      ur[c] = R(u[((long long)er * NV + v) * P + nr]);
      gg[c] = R(tb.liftR[dir] * w[((long long)e * NV + v) * P + nl] +
                tb.liftL[dir] * w[((long long)er * NV + v) * P + nr]);
    }
    if (sf == kSLLF && sizeof(R) == 8)
      llf_rev<R, D>(ul, ur, gg, R(g.gamma), R(g.gm1), gl, gr);
    else
      pair_vjp<R, D>(0, sf, true, ul, ur, gg, R(g.gamma), R(g.gm1), R(g.gm1inv), gl, gr);
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const int v = nf_index<D>(dir, c);
      fb[((long long)((dir * 2 + 0) * NV + v) * nelem + e) * NF + l] = (double)gl[c];
      fb[((long long)((dir * 2 + 1) * NV + v) * nelem + e) * NF + l] = (double)gr[c];
    }
  }
}

template <int D, int N, typename R>
__global__ void vjp_face_kernel(const double* __restrict__ u, const double* __restrict__ w,
                                double* __restrict__ fb, Geom g, Tables<double> tb, int sf) {
  if (blockIdx.y == 0) vjp_face_body<D, N, R, 0>(u, w, fb, g, tb, sf);
  else if (blockIdx.y == 1) vjp_face_body<D, N, R, 1>(u, w, fb, g, tb, sf);
  else vjp_face_body<D, N, R, (D == 3 ? 2 : 1)>(u, w, fb, g, tb, sf);
}

template <int D, int N, typename R, int EPB>
__global__ void __launch_bounds__(EPB* Shape<D, N>::LINES)
    vjp_volume_kernel(const double* __restrict__ u, const double* __restrict__ w,
                      double* __restrict__ ubar, const double* __restrict__ fb, Geom g,
                      Tables<double> tb, int vf) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, P = S::P, NV = S::NV, LINES = S::LINES;
  extern __shared__ __align__(16) unsigned char dg_smem[];
  double(*su)[NV][P] = reinterpret_cast<double(*)[NV][P]>(dg_smem);
  double(*sw)[NV][P] = su + EPB;
  double(*sb)[NV][P] = sw + EPB;
  __shared__ int s_left[EPB][3];
  const int e0 = blockIdx.x * EPB;
  const int nelem = (int)g.nelem;
  if (threadIdx.x < EPB && e0 + (int)threadIdx.x < nelem) {
    const int el = threadIdx.x, e = e0 + el;
    const int x = e % g.n[0], r = e / g.n[0], y = r % g.n[1], z = r / g.n[1];
    s_left[el][0] = elem_index(g, x == 0 ? g.n[0] - 1 : x - 1, y, z);
    s_left[el][1] = elem_index(g, x, y == 0 ? g.n[1] - 1 : y - 1, z);
    s_left[el][2] = (D == 3) ? elem_index(g, x, y, z == 0 ? g.n[2] - 1 : z - 1) : 0;
  }
  for (int t = threadIdx.x; t < EPB * NV * P; t += blockDim.x) {
    const int el = t / (NV * P), r = t % (NV * P);
    const int e = e0 + el;
    if (e >= nelem) continue;
    su[el][r / P][r % P] = u[(long long)e * NV * P + r];
    sw[el][r / P][r % P] = w[(long long)e * NV * P + r];
    sb[el][r / P][r % P] = 0.0;
  }
  __syncthreads();
  const int el = threadIdx.x / LINES, l = threadIdx.x % LINES;
  const bool active = (e0 + el) < nelem;
#pragma unroll 1
  for (int dir = 0; dir < D; ++dir) {
    if (active) {
#pragma unroll 1
      for (int a = 0; a < NP; ++a) {
        const int na = line_node_rt<D, N>(dir, l, a);
#pragma unroll 1
        for (int b = a + 1; b < NP; ++b) {
          const int nb = line_node_rt<D, N>(dir, l, b);
          const double dab = tb.Ds[dir][a][b], dba = tb.Ds[dir][b][a];
          R ua[NV], ub[NV], gg[NV], ga[NV], gb[NV];
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            const int v = nf_index<D>(dir, c);
            ua[c] = R(su[el][v][na]);
            ub[c] = R(su[el][v][nb]);
            gg[c] = R(dab * sw[el][v][na] + dba * sw[el][v][nb]);
          }
          pair_vjp<R, D>(vf, 0, false, ua, ub, gg, R(g.gamma), R(g.gm1), R(g.gm1inv), ga, gb);
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            const int v = nf_index<D>(dir, c);
            sb[el][v][na] += (double)ga[c];
            sb[el][v][nb] += (double)gb[c];
          }
        }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
    const int ell = t / P, node = t % P;
    const int e = e0 + ell;
    if (e >= nelem) continue;
    const int c[3] = {node % NP, (node / NP) % NP, node / (NP * NP)};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double val = sb[ell][v][node];
#pragma unroll
      for (int dir = 0; dir < D; ++dir) {
        const int lf = (D == 2) ? ((dir == 0) ? c[1] : c[0])
                                : (dir == 0) ? (c[1] + NP * c[2])
                                : (dir == 1) ? (c[0] + NP * c[2]) : (c[0] + NP * c[1]);
        if (c[dir] == N) val += fb[((long long)((dir * 2 + 0) * NV + v) * nelem + e) * LINES + lf];
        if (c[dir] == 0)
          val += fb[((long long)((dir * 2 + 1) * NV + v) * nelem + s_left[ell][dir]) * LINES + lf];
      }
      ubar[((long long)e * NV + v) * P + node] = val;
    }
  }
}

// Ranocha's volume flux in reverse mode: the primitives of every node once
// per element in shared memory, the pair adjoints (ranocha_pair_rev)
// accumulated as adjoints of the primitives, and in the epilogue one
// conversion per node to the adjoint of the conserved variables,
//   ubar_rho = rhobar - sum_k vbar_k v_k / rho + pbar (gamma-1) |v|^2 / 2,
//   ubar_m_k = vbar_k / rho - pbar (gamma-1) v_k,   ubar_E = pbar (gamma-1),
// plus the face contributions.
template <int D, int N, typename R, int EPB>
__global__ void __launch_bounds__(EPB* Shape<D, N>::LINES)
    vjp_volume_rev_kernel(const double* __restrict__ u, const double* __restrict__ w,
                          double* __restrict__ ubar, const double* __restrict__ fb, Geom g,
                          Tables<double> tb) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, P = S::P, NV = S::NV, LINES = S::LINES;
  extern __shared__ __align__(16) unsigned char dg_smem[];
  double(*sq)[NV][P] = reinterpret_cast<double(*)[NV][P]>(dg_smem);  // rho, v, p
  double(*sw)[NV][P] = sq + EPB;
  double(*sb)[NV][P] = sw + EPB;  // adjoints of rho, v, p
  __shared__ int s_left[EPB][3];
  const int e0 = blockIdx.x * EPB;
  const int nelem = (int)g.nelem;
  if (threadIdx.x < EPB && e0 + (int)threadIdx.x < nelem) {
    const int el = threadIdx.x, e = e0 + el;
    const int x = e % g.n[0], r = e / g.n[0], y = r % g.n[1], z = r / g.n[1];
    s_left[el][0] = elem_index(g, x == 0 ? g.n[0] - 1 : x - 1, y, z);
    s_left[el][1] = elem_index(g, x, y == 0 ? g.n[1] - 1 : y - 1, z);
    s_left[el][2] = (D == 3) ? elem_index(g, x, y, z == 0 ? g.n[2] - 1 : z - 1) : 0;
  }
  for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
    const int el = t / P, node = t % P;
    const int e = e0 + el;
    if (e >= nelem) continue;
    double c[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      c[v] = u[((long long)e * NV + v) * P + node];
      sw[el][v][node] = w[((long long)e * NV + v) * P + node];
      sb[el][v][node] = 0.0;
    }
    const Prim<double, D> q = cons2prim<double, D>(c, g.gm1);
    sq[el][0][node] = q.rho;
#pragma unroll
    for (int k = 0; k < D; ++k) sq[el][1 + k][node] = q.v[k];
    sq[el][D + 1][node] = q.p;
  }
  __syncthreads();
  const int el = threadIdx.x / LINES, l = threadIdx.x % LINES;
  const bool active = (e0 + el) < nelem;
  const R gm1inv = R(g.gm1inv);
#pragma unroll 1
  for (int dir = 0; dir < D; ++dir) {
    if (active) {
#pragma unroll 1
      for (int a = 0; a < NP; ++a) {
        const int na = line_node_rt<D, N>(dir, l, a);
#pragma unroll 1
        for (int b = a + 1; b < NP; ++b) {
          const int nb = line_node_rt<D, N>(dir, l, b);
          const double dab = tb.Ds[dir][a][b], dba = tb.Ds[dir][b][a];
          R qa[NV], qb[NV], gg[NV], ga[NV], gb[NV];
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            const int v = nf_index<D>(dir, c);
            qa[c] = R(sq[el][v][na]);
            qb[c] = R(sq[el][v][nb]);
            gg[c] = R(dab * sw[el][v][na] + dba * sw[el][v][nb]);
            ga[c] = R(0);
            gb[c] = R(0);
          }
          ranocha_pair_rev<R, D>(qa, qb, gg, gm1inv, ga, gb);
#pragma unroll
          for (int c = 0; c < NV; ++c) {
            const int v = nf_index<D>(dir, c);
            sb[el][v][na] += (double)ga[c];
            sb[el][v][nb] += (double)gb[c];
          }
        }
      }
    }
    __syncthreads();
  }
  const double gm1 = g.gm1;
  for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
    const int ell = t / P, node = t % P;
    const int e = e0 + ell;
    if (e >= nelem) continue;
    const double rho = sq[ell][0][node], pb = sb[ell][D + 1][node];
    const double irho = 1.0 / rho;
    double val[NV], v2 = 0.0, rb = sb[ell][0][node];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double vk = sq[ell][1 + k][node], vbk = sb[ell][1 + k][node];
      v2 += vk * vk;
      rb -= vbk * vk * irho;
      val[1 + k] = vbk * irho - pb * gm1 * vk;
    }
    val[0] = rb + pb * gm1 * 0.5 * v2;
    val[D + 1] = pb * gm1;
    const int c[3] = {node % NP, (node / NP) % NP, node / (NP * NP)};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double acc = val[v];
#pragma unroll
      for (int dir = 0; dir < D; ++dir) {
        const int lf = (D == 2) ? ((dir == 0) ? c[1] : c[0])
                                : (dir == 0) ? (c[1] + NP * c[2])
                                : (dir == 1) ? (c[0] + NP * c[2]) : (c[0] + NP * c[1]);
        if (c[dir] == N) acc += fb[((long long)((dir * 2 + 0) * NV + v) * nelem + e) * LINES + lf];
        if (c[dir] == 0)
          acc += fb[((long long)((dir * 2 + 1) * NV + v) * nelem + s_left[ell][dir]) * LINES + lf];
      }
      ubar[((long long)e * NV + v) * P + node] = acc;
    }
  }
}

// elements per CTA of the VJP volume kernels (one thread per element line):
// about 64 threads, unless their warps would leave more than a tenth of the
// lanes idle (a warp's FP64 instruction costs the same whatever its active
// lanes); then the count of at most 256 threads and 96 KB of shared memory
// that fills the warps best
template <int LINES, int PER>
constexpr int vjp_epb() {
  constexpr int byt = (64 / LINES) > 0 ? (64 / LINES) : 1;
  constexpr int bys = (98304 / PER) > 0 ? (98304 / PER) : 1;
  constexpr int base = byt < bys ? byt : bys;
  auto fill = [](int t) { return (double)t / (32.0 * ((t + 31) / 32)); };
  if (fill(base * LINES) >= 0.9) return base;
  int best = base;
  for (int e = 1; e * LINES <= 256 && e * PER <= 98304; ++e)
    if (fill(e * LINES) > fill(best * LINES) + 0.01) best = e;
  return best;
}

template <int D, int N, typename R>
cudaError_t launch_vjp_dn(const double* u, const double* w, double* ubar, double* fb,
                          const Geom& g, const Tables<double>& tb, int vf, int sf,
                          cudaStream_t st) {
  using S = Shape<D, N>;
  constexpr int PER = 3 * S::NV * S::P * (int)sizeof(double);
  constexpr int EPB = vjp_epb<S::LINES, PER>();
  constexpr int SM = EPB * PER;
  {
    const long long total = g.nelem * S::LINES;
    long long blocks = (total + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    vjp_face_kernel<D, N, R><<<dim3((unsigned)blocks, D), 128, 0, st>>>(u, w, fb, g, tb, sf);
  }
  const long long grid = (g.nelem + EPB - 1) / EPB;
  cudaError_t e;
  if (vf == kVRanocha && sizeof(R) == 8) {
    if ((e = allow_smem(vjp_volume_rev_kernel<D, N, R, EPB>, SM)) != cudaSuccess) return e;
    vjp_volume_rev_kernel<D, N, R, EPB><<<(unsigned)grid, EPB * S::LINES, SM, st>>>(u, w, ubar,
                                                                                  fb, g, tb);
    return cudaGetLastError();
  }
  if ((e = allow_smem(vjp_volume_kernel<D, N, R, EPB>, SM)) != cudaSuccess) return e;
  vjp_volume_kernel<D, N, R, EPB><<<(unsigned)grid, EPB * S::LINES, SM, st>>>(u, w, ubar, fb, g,
                                                                              tb, vf);
  return cudaGetLastError();
}

template <int D, typename R>
cudaError_t launch_vjp_d(int N, const double* u, const double* w, double* ubar, double* fb,
                         const Geom& g, const Tables<double>& tb, int vf, int sf,
                         cudaStream_t st) {
  switch (N) {
    case 1: return launch_vjp_dn<D, 1, R>(u, w, ubar, fb, g, tb, vf, sf, st);
    case 2: return launch_vjp_dn<D, 2, R>(u, w, ubar, fb, g, tb, vf, sf, st);
    case 3: return launch_vjp_dn<D, 3, R>(u, w, ubar, fb, g, tb, vf, sf, st);
    case 4: return launch_vjp_dn<D, 4, R>(u, w, ubar, fb, g, tb, vf, sf, st);
    case 5: return launch_vjp_dn<D, 5, R>(u, w, ubar, fb, g, tb, vf, sf, st);
    case 6: return launch_vjp_dn<D, 6, R>(u, w, ubar, fb, g, tb, vf, sf, st);
    case 7: return launch_vjp_dn<D, 7, R>(u, w, ubar, fb, g, tb, vf, sf, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
