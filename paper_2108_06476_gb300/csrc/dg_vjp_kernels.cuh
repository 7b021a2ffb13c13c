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

template <int D, int N, typename R>
cudaError_t launch_vjp_dn(const double* u, const double* w, double* ubar, double* fb,
                          const Geom& g, const Tables<double>& tb, int vf, int sf,
                          cudaStream_t st) {
  using S = Shape<D, N>;
  constexpr int PER = 3 * S::NV * S::P * (int)sizeof(double);
  constexpr int BYT = (64 / S::LINES) > 0 ? (64 / S::LINES) : 1;
  constexpr int BYS = (98304 / PER) > 0 ? (98304 / PER) : 1;
  constexpr int EPB = BYT < BYS ? BYT : BYS;
  constexpr int SM = EPB * PER;
  {
    const long long total = g.nelem * S::LINES;
    long long blocks = (total + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    vjp_face_kernel<D, N, R><<<dim3((unsigned)blocks, D), 128, 0, st>>>(u, w, fb, g, tb, sf);
  }
  cudaError_t e = allow_smem(vjp_volume_kernel<D, N, R, EPB>, SM);
  if (e != cudaSuccess) return e;
  const long long grid = (g.nelem + EPB - 1) / EPB;
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
