// The two kernels of one rhs evaluation (Sec. 2.1 DGSEM, Eq. (1) with s = 0):
//
//  surface_kernel: one thread per face node; evaluates the surface flux F*
//    between the trace u_L (node N of the left element) and u_R (node 0 of
//    the right element) of every interface and stores it in the face buffer
//    fs[dir][v][e_left][l] (l = face-node index, see line_node).
//
//  volume_kernel: one CTA per EPB elements, one thread per element line.
//    Prologue: conserved -> primitive at every node into shared memory.
//    Per direction: each thread walks its line's N(N+1)/2 node pairs once,
//    evaluating f#(u_a, u_b) a single time for both nodes, since f# is
//    symmetric and the split-form matrix has a zero diagonal:
//      du_a += Ds[a][b] f#(u_a, u_b),  du_b += Ds[b][a] f#(u_a, u_b).
//    Epilogue: lifting of the face fluxes at the element's boundary nodes,
//    du += liftR F*_R (node N) + liftL F*_L (node 0) per direction, and one
//    coalesced store of du.
#pragma once
#include "dg_device.cuh"

namespace dg {

template <int D, int N, typename R>
__global__ void surface_kernel(const double* __restrict__ u, R* __restrict__ fs, Geom g, int sf) {
  using S = Shape<D, N>;
  constexpr int NV = S::NV, P = S::P, NF = S::LINES;
  const int dir = blockIdx.y;
  const long long total = g.nelem * NF;
  const R gamma = R(g.gamma), gm1 = R(g.gamma - 1.0), gm1inv = R(1.0 / (g.gamma - 1.0));
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / NF;
    const int l = (int)(t % NF);
    const long long er = neighbour(g, e, dir, +1);
    const int nl = line_node_rt<D, N>(dir, l, N), nr = line_node_rt<D, N>(dir, l, 0);
    R cl[NV], cr[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      cl[v] = R(u[(e * NV + v) * P + nl]);
      cr[v] = R(u[(er * NV + v) * P + nr]);
    }
    const Prim<R, D> ql = cons2prim<R, D>(cl, gm1), qr = cons2prim<R, D>(cr, gm1);
    R f[NV];
    if (dir == 0) surface_flux_dir<R, D, 0>(sf, cl, cr, ql, qr, gamma, gm1inv, f);
    else if (dir == 1) surface_flux_dir<R, D, 1>(sf, cl, cr, ql, qr, gamma, gm1inv, f);
    else surface_flux_dir<R, D, (D == 3 ? 2 : 1)>(sf, cl, cr, ql, qr, gamma, gm1inv, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) fs[((long long)(dir * NV + v) * g.nelem + e) * NF + l] = f[v];
  }
}

// One direction of the flux-differencing volume term for the line owned by
// this thread; adds the line's contributions into the shared accumulators.
template <int D, int N, typename R, int VF, int DIR, int EPB>
__device__ __forceinline__ void volume_direction(R (*sp)[D + 2][Shape<D, N>::P],
                                                 R (*sa)[D + 2][Shape<D, N>::P], int el, int l,
                                                 const Tables<R>& tb, R gm1inv) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, NV = S::NV;
  Prim<R, D> q[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int node = line_node<D, N, DIR>(l, a);
    q[a].rho = sp[el][0][node];
#pragma unroll
    for (int k = 0; k < D; ++k) q[a].v[k] = sp[el][1 + k][node];
    q[a].p = sp[el][D + 1][node];
  }
  R acc[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[a][v] = R(0);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = a + 1; b < NP; ++b) {
      R f[NV];
      volume_flux<VF, R, D, DIR>(q[a], q[b], gm1inv, f);
      const R dab = tb.Ds[DIR][a][b], dba = tb.Ds[DIR][b][a];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[a][v] += dab * f[v];
        acc[b][v] += dba * f[v];
      }
    }
  }
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int node = line_node<D, N, DIR>(l, a);
#pragma unroll
    for (int v = 0; v < NV; ++v) sa[el][v][node] += acc[a][v];
  }
}

template <int D, int N, typename R, int VF, int EPB>
__global__ void __launch_bounds__(EPB* Shape<D, N>::LINES)
    volume_kernel(const double* __restrict__ u, R* __restrict__ du, const R* __restrict__ fs,
                  Geom g, Tables<R> tb, unsigned* __restrict__ err) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, P = S::P, NV = S::NV, LINES = S::LINES;
  __shared__ R sp[EPB][NV][P];  // primitives rho, v_1..v_d, p
  __shared__ R sa[EPB][NV][P];  // accumulated volume terms
  const long long e0 = (long long)blockIdx.x * EPB;
  const R gm1 = R(g.gamma - 1.0), gm1inv = R(1.0 / (g.gamma - 1.0));
  unsigned bad = 0;
  for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
    const int el = t / P, node = t % P;
    const long long e = e0 + el;
    if (e < g.nelem) {
      R c[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) c[v] = R(u[(e * NV + v) * P + node]);
      const Prim<R, D> q = cons2prim<R, D>(c, gm1);
      bad |= prim_check(q);
      sp[el][0][node] = q.rho;
#pragma unroll
      for (int k = 0; k < D; ++k) sp[el][1 + k][node] = q.v[k];
      sp[el][D + 1][node] = q.p;
#pragma unroll
      for (int v = 0; v < NV; ++v) sa[el][v][node] = R(0);
    }
  }
  if (bad) atomicOr(err, bad);
  __syncthreads();
  const int el = threadIdx.x / LINES, l = threadIdx.x % LINES;
  const bool active = (e0 + el) < g.nelem;
  if (active) volume_direction<D, N, R, VF, 0, EPB>(sp, sa, el, l, tb, gm1inv);
  __syncthreads();
  if (active) volume_direction<D, N, R, VF, 1, EPB>(sp, sa, el, l, tb, gm1inv);
  if (D == 3) {
    __syncthreads();
    if (active) volume_direction<D, N, R, VF, (D == 3 ? 2 : 1), EPB>(sp, sa, el, l, tb, gm1inv);
  }
  __syncthreads();
  // epilogue: lifting of the surface fluxes, then the store
  for (int t = threadIdx.x; t < EPB * P; t += blockDim.x) {
    const int ell = t / P, node = t % P;
    const long long e = e0 + ell;
    if (e >= g.nelem) continue;
    int c[3] = {node % NP, (node / NP) % NP, node / (NP * NP)};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      R val = sa[ell][v][node];
#pragma unroll
      for (int dir = 0; dir < D; ++dir) {
        // face-node index: the node's other coordinates, first one fastest
        const int lf = (dir == 0) ? (c[1] + NP * c[2]) : (dir == 1) ? (c[0] + NP * c[2])
                                                                    : (c[0] + NP * c[1]);
        const int lf2 = (D == 2) ? ((dir == 0) ? c[1] : c[0]) : lf;
        if (c[dir] == N)
          val += tb.liftR[dir] * fs[((long long)(dir * NV + v) * g.nelem + e) * LINES + lf2];
        if (c[dir] == 0) {
          const long long el_ = neighbour(g, e, dir, -1);
          val += tb.liftL[dir] * fs[((long long)(dir * NV + v) * g.nelem + el_) * LINES + lf2];
        }
      }
      du[(e * NV + v) * P + node] = val;
    }
  }
}

// elements per CTA: about 128 threads, shared memory <= 40 KB
template <int D, int N, typename R>
struct Launch {
  static constexpr int LINES = Shape<D, N>::LINES;
  static constexpr int BY_THREADS = (128 / LINES) > 0 ? (128 / LINES) : 1;
  static constexpr int PER_ELEM = 2 * Shape<D, N>::NV * Shape<D, N>::P * (int)sizeof(R);
  static constexpr int BY_SMEM = (40960 / PER_ELEM) > 0 ? (40960 / PER_ELEM) : 1;
  static constexpr int EPB = BY_THREADS < BY_SMEM ? BY_THREADS : BY_SMEM;
};

// parts: bit 0 = surface kernel, bit 1 = volume kernel (both for an rhs)
template <int D, int N, typename R>
cudaError_t launch_rhs_dn(const double* u, R* du, R* fs, const Geom& g, const Tables<R>& tb,
                          int vf, int sf, unsigned* err, cudaStream_t st, int parts) {
  using L = Launch<D, N, R>;
  constexpr int EPB = L::EPB;
  if (parts & 1) {
    const long long total = g.nelem * Shape<D, N>::LINES;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    surface_kernel<D, N, R><<<dim3((unsigned)blocks, D), 256, 0, st>>>(u, fs, g, sf);
  }
  if (!(parts & 2)) return cudaGetLastError();
  const long long grid = (g.nelem + EPB - 1) / EPB;
  const int threads = EPB * L::LINES;
  if (vf == kVRanocha)
    volume_kernel<D, N, R, kVRanocha, EPB><<<(unsigned)grid, threads, 0, st>>>(u, du, fs, g, tb, err);
  else if (vf == kVChandrashekar)
    volume_kernel<D, N, R, kVChandrashekar, EPB><<<(unsigned)grid, threads, 0, st>>>(u, du, fs, g, tb, err);
  else
    volume_kernel<D, N, R, kVCentral, EPB><<<(unsigned)grid, threads, 0, st>>>(u, du, fs, g, tb, err);
  return cudaGetLastError();
}

template <int D, typename R>
cudaError_t launch_rhs_d(int N, const double* u, R* du, R* fs, const Geom& g, const Tables<R>& tb,
                         int vf, int sf, unsigned* err, cudaStream_t st, int parts) {
  switch (N) {
    case 1: return launch_rhs_dn<D, 1, R>(u, du, fs, g, tb, vf, sf, err, st, parts);
    case 2: return launch_rhs_dn<D, 2, R>(u, du, fs, g, tb, vf, sf, err, st, parts);
    case 3: return launch_rhs_dn<D, 3, R>(u, du, fs, g, tb, vf, sf, err, st, parts);
    case 4: return launch_rhs_dn<D, 4, R>(u, du, fs, g, tb, vf, sf, err, st, parts);
    case 5: return launch_rhs_dn<D, 5, R>(u, du, fs, g, tb, vf, sf, err, st, parts);
    case 6: return launch_rhs_dn<D, 6, R>(u, du, fs, g, tb, vf, sf, err, st, parts);
    case 7: return launch_rhs_dn<D, 7, R>(u, du, fs, g, tb, vf, sf, err, st, parts);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
