// FP32 kernels of one rhs evaluation in perturbation form (dg_f32.cuh):
//
//  ref_kernel: one thread per element writes its FP32 reference (rho0, v0,
//    p0) from the element's central node into the library's reference buffer.
//    Every later kernel of the stage reads references from that buffer
//    (never from u, which the fused volume kernel updates in place).
//
//  surface_kernel32: one thread per face node; both traces are taken as
//    deviations from the LEFT element's reference and the kernel stores
//    F* - f(ref_left) in the face buffer fs[dir][v][e_left][l].
//
//  volume_kernel32: one CTA per EPB elements, one thread per element line,
//    the same organisation as the FP64 volume kernel (pair halving, lifting at
//    the line ends of each direction phase, fused stage update). The
//    two-point fluxes are f#(u_a, u_b) - f(ref_e); at the right face of each
//    line the stored flux is already relative to this element's reference,
//    at the left face it is relative to the left neighbour's and the kernel
//    adds fl32(f(ref_left) - f(ref_e)), formed in FP64 once per element and
//    direction. Because the split-form operator annihilates a constant flux
//    together with the lifting, du is unchanged by these subtractions.
#pragma once
#include "dg_f32.cuh"

namespace dg {

template <int D, int N, int VF>
__device__ __forceinline__ void volume_direction32(int dir,
                                                   float (*sp)[3 + 2 * D][Shape<D, N>::P],
                                                   float (*sa)[D + 2][Shape<D, N>::P], int el,
                                                   int l, const Tables<float>& tb, float gm1inv,
                                                   float ggm1, const float* __restrict__ fs,
                                                   int nelem, int e, int eleft,
                                                   const float* rref, const float* dc) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, NV = S::NV;
  const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  int node[NP];
  DNode<D> q[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    node[a] = line_node_rt<D, N>(dir, l, a);
    const int nd = node[a];
    q[a].rho = sp[el][0][nd];
    q[a].drho = sp[el][1][nd];
    q[a].dp = sp[el][2][nd];
    q[a].v[0] = sp[el][3 + dir][nd];
    q[a].dv[0] = sp[el][3 + D + dir][nd];
    q[a].v[1] = sp[el][3 + t1][nd];
    q[a].dv[1] = sp[el][3 + D + t1][nd];
    if (D == 3) {
      q[a].v[D - 1] = sp[el][3 + t2][nd];
      q[a].dv[D - 1] = sp[el][3 + D + t2][nd];
    }
  }
  // the line's two face fluxes, loaded before the pair loop so that their
  // latency overlaps it
  int comp[NV];
  comp[0] = 0;
  comp[1] = 1 + dir;
  comp[2] = 1 + t1;
  if (D == 3) comp[D] = 1 + t2;
  comp[D + 1] = D + 1;
  float fR[NV], fL[NV];
  {
    const long long base = (long long)nelem * S::LINES;
    const long long oR = (long long)e * S::LINES + l;
    const long long oL = (long long)eleft * S::LINES + l;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const long long row = (long long)(dir * NV + comp[c]) * base;
      fR[c] = fs[row + oR];
      fL[c] = fs[row + oL] + dc[comp[c]];
    }
  }
  const DRef<D> rf = dir_ref<D>(rref[0], rref + 1, rref[D + 1], dir);
  // strong form: du_a = sum_b Ds_ab (f#_ab - F_a) + lift (F* - F_a) with F_a
  // the node's own flux (the identity sum_b Ds_ab = -lift_a), so that no
  // partial sum carries the node's offset from the reference times the
  // large entries of Dt
  float Fn[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a) delta_phys_flux<D>(q[a], rf, ggm1, Fn[a]);
  float acc[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[a][v] = 0.0f;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = a + 1; b < NP; ++b) {
      const float dab = tb.Ds[dir][a][b], dba = tb.Ds[dir][b][a];
      if (VF == kVCentral) {
        // f#_ab - F_a = (F_b - F_a)/2 = -(f#_ab - F_b)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float h = 0.5f * (Fn[b][v] - Fn[a][v]);
          acc[a][v] = fmaf(dab, h, acc[a][v]);
          acc[b][v] = fmaf(-dba, h, acc[b][v]);
        }
      } else {
        float f[NV];
        delta_pair<VF, D>(q[a], q[b], rf, gm1inv, f);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          acc[a][v] = fmaf(dab, f[v] - Fn[a][v], acc[a][v]);
          acc[b][v] = fmaf(dba, f[v] - Fn[b][v], acc[b][v]);
        }
      }
    }
  }
  // lifting at the line ends; the left face's flux is relative to the left
  // neighbour's reference, corrected by dc = fl32(f(ref_left) - f(ref_e))
  {
    const float lr = tb.liftR[dir], ll = tb.liftL[dir];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      acc[N][c] = fmaf(lr, fR[c] - Fn[N][c], acc[N][c]);
      acc[0][c] = fmaf(ll, fL[c] - Fn[0][c], acc[0][c]);
    }
  }
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int nd = node[a];
    sa[el][0][nd] += acc[a][0];
    sa[el][1 + dir][nd] += acc[a][1];
    sa[el][1 + t1][nd] += acc[a][2];
    if (D == 3) sa[el][1 + t2][nd] += acc[a][D];
    sa[el][D + 1][nd] += acc[a][D + 1];
  }
}

// Degrees from kRows32FromN up: volume_direction32 with the row node a of
// the pair loop as a loop value (one flux body per partner node b instead of
// one per pair) and the partner's staged deviations read from shared memory
// for each pair; the row's running sums and own flux are taken out of the
// register arrays and put back, so every node's sum takes its terms in the
// same order: bitwise the result of volume_direction32 (see
// volume_direction_rows). On GB300 it raises the FP32 rhs of 3D N = 4, 5,
// 6 and 7 by 8%, 12%, 23% and 25%; N = 3 keeps the line-held form (7% faster
// there).
constexpr int kRows32FromN = 4;

template <int D, int N, int VF>
__device__ __forceinline__ void volume_direction32_rows(
    int dir, float (*sp)[3 + 2 * D][Shape<D, N>::P], float (*sa)[D + 2][Shape<D, N>::P], int el,
    int l, const Tables<float>& tb, float gm1inv, float ggm1, const float* __restrict__ fs,
    int nelem, int e, int eleft, const float* rref, const float* dc) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, NV = S::NV;
  const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  const int n0 = line_node_rt<D, N>(dir, l, 0);
  const int ns = line_node_rt<D, N>(dir, l, 1) - n0;  // node stride along the line
  auto stage = [&](int a) {
    const int nd = n0 + a * ns;
    DNode<D> q;
    q.rho = sp[el][0][nd];
    q.drho = sp[el][1][nd];
    q.dp = sp[el][2][nd];
    q.v[0] = sp[el][3 + dir][nd];
    q.dv[0] = sp[el][3 + D + dir][nd];
    q.v[1] = sp[el][3 + t1][nd];
    q.dv[1] = sp[el][3 + D + t1][nd];
    if (D == 3) {
      q.v[D - 1] = sp[el][3 + t2][nd];
      q.dv[D - 1] = sp[el][3 + D + t2][nd];
    }
    return q;
  };
  int comp[NV];
  comp[0] = 0;
  comp[1] = 1 + dir;
  comp[2] = 1 + t1;
  if (D == 3) comp[D] = 1 + t2;
  comp[D + 1] = D + 1;
  float fR[NV], fL[NV];
  {
    const long long base = (long long)nelem * S::LINES;
    const long long oR = (long long)e * S::LINES + l;
    const long long oL = (long long)eleft * S::LINES + l;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const long long row = (long long)(dir * NV + comp[c]) * base;
      fR[c] = fs[row + oR];
      fL[c] = fs[row + oL] + dc[comp[c]];
    }
  }
  const DRef<D> rf = dir_ref<D>(rref[0], rref + 1, rref[D + 1], dir);
  float Fn[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const DNode<D> q = stage(a);
    delta_phys_flux<D>(q, rf, ggm1, Fn[a]);
  }
  float acc[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[a][v] = 0.0f;
#pragma unroll 1
  for (int a = 0; a < NP - 1; ++a) {
    const DNode<D> qa = stage(a);
    float ra[NV], Fa[NV];
#pragma unroll
    for (int k = 0; k < NP - 1; ++k)
      if (k == a)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          ra[v] = acc[k][v];
          Fa[v] = Fn[k][v];
        }
#pragma unroll
    for (int b = 1; b < NP; ++b) {
      if (b > a) {
        const float dab = tb.Ds[dir][a][b], dba = tb.Ds[dir][b][a];
        if (VF == kVCentral) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const float h = 0.5f * (Fn[b][v] - Fa[v]);
            ra[v] = fmaf(dab, h, ra[v]);
            acc[b][v] = fmaf(-dba, h, acc[b][v]);
          }
        } else {
          const DNode<D> qb = stage(b);
          float f[NV];
          delta_pair<VF, D>(qa, qb, rf, gm1inv, f);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            ra[v] = fmaf(dab, f[v] - Fa[v], ra[v]);
            acc[b][v] = fmaf(dba, f[v] - Fn[b][v], acc[b][v]);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NP - 1; ++k)
      if (k == a)
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[k][v] = ra[v];
  }
  {
    const float lr = tb.liftR[dir], ll = tb.liftL[dir];
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      acc[N][c] = fmaf(lr, fR[c] - Fn[N][c], acc[N][c]);
      acc[0][c] = fmaf(ll, fL[c] - Fn[0][c], acc[0][c]);
    }
  }
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int nd = n0 + a * ns;
    sa[el][0][nd] += acc[a][0];
    sa[el][1 + dir][nd] += acc[a][1];
    sa[el][1 + t1][nd] += acc[a][2];
    if (D == 3) sa[el][1 + t2][nd] += acc[a][D];
    sa[el][D + 1][nd] += acc[a][D + 1];
  }
}

// One batch of `count` (<= MAXE) elements from e0 (see volume_batch);
// fz.ref holds the references of every element of the mesh. smem: count x
// (3 + 2D) staged slots and count x (D + 2) accumulators (FP32), then, from
// the next 16-byte boundary, count x (D + 2) x P doubles for the RK register
// (dynamic size: volume32_smem).
template <int D, int N>
constexpr int volume32_smem(int count) {
  return ((4 * count * (3 + 2 * D + D + 2) * Shape<D, N>::P + 15) & ~15) +
         8 * count * (D + 2) * Shape<D, N>::P;
}

template <int D, int N, int VF, int MAXE>
__device__ __forceinline__ void volume_batch32(double* u, float* __restrict__ du,
                                               const float* __restrict__ fs, const Geom& g,
                                               const Tables<float>& tb,
                                               unsigned* __restrict__ err, const StageFuse& fz,
                                               int e0, int count, unsigned char* smem) {
  using S = Shape<D, N>;
  constexpr int P = S::P, NV = S::NV, LINES = S::LINES;
  constexpr int NC = 3 + 2 * D;  // rho, drho, dp, v[D], dv[D]
  float(*sp)[NC][P] = reinterpret_cast<float(*)[NC][P]>(smem);
  float(*sa)[NV][P] = reinterpret_cast<float(*)[NV][P]>(smem + sizeof(float) * count * NC * P);
  __shared__ int s_left[MAXE][3];
  __shared__ float s_ref[MAXE][D + 2];
  __shared__ double s_E0[MAXE];
  __shared__ float s_dc[MAXE][D][NV];
  const int nelem = (int)g.nelem;
  const float* __restrict__ ref = fz.ref;
  // one thread per (element, direction): the left neighbour and the face
  // correction fl32(f(ref_left) - f(ref_e)) in FP64; every reference load is
  // issued at once
  if ((int)threadIdx.x < count * D) {
    const int el = threadIdx.x / D, dir = threadIdx.x % D, e = e0 + el;
    const int x = e % g.n[0], r = e / g.n[0], y = r % g.n[1], z = r / g.n[1];
    int left;
    if (dir == 0) left = elem_index(g, x == 0 ? g.n[0] - 1 : x - 1, y, z);
    else if (dir == 1) left = elem_index(g, x, y == 0 ? g.n[1] - 1 : y - 1, z);
    else left = elem_index(g, x, y, z == 0 ? g.n[2] - 1 : z - 1);
    s_left[el][dir] = left;
    const float* own = ref + (long long)e * NV;
    double co[NV], cl[NV];
    ref_flux64<D>(own, dir, g.gamma, g.gm1inv, co);
    ref_flux64<D>(ref + (long long)left * NV, dir, g.gamma, g.gm1inv, cl);
#pragma unroll
    for (int v = 0; v < NV; ++v) s_dc[el][dir][v] = (float)(cl[v] - co[v]);
    if (dir == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) s_ref[el][v] = own[v];
      s_E0[el] = fz.refE[e];
    }
  }
  // the RK register of the batch (read by the fused epilogue) is staged in
  // shared memory together with the state loads below
  double* sk = reinterpret_cast<double*>(
      smem + ((sizeof(float) * count * (NC + NV) * P + 15) & ~(size_t)15));
  const bool stage_k = fz.k && fz.a != 0.0;
  __syncthreads();
  const float gm1f = (float)g.gm1;
  unsigned bad = 0;
  for (int t = threadIdx.x; t < count * P; t += blockDim.x) {
    const int el = t / P, node = t % P;
    const int e = e0 + el;
    double c[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = u[((long long)e * NV + v) * P + node];
    if (stage_k) {
#pragma unroll
      for (int v = 0; v < NV; ++v) sk[(el * NV + v) * P + node] = fz.k[((long long)e * NV + v) * P + node];
    }
    DNode<D> q;
    delta_node<D>(c, s_ref[el][0], &s_ref[el][1], s_E0[el], gm1f, q);
    const float p = s_ref[el][D + 1] + q.dp;
    if (!(q.rho > 0.0f)) bad |= kErrRho;
    if (!(p > 0.0f)) bad |= kErrP;
    if (!isfinite(q.rho) || !isfinite(p)) bad |= kErrNaN;
    sp[el][0][node] = q.rho;
    sp[el][1][node] = q.drho;
    sp[el][2][node] = q.dp;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      sp[el][3 + k][node] = q.v[k];
      sp[el][3 + D + k][node] = q.dv[k];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) sa[el][k][node] = 0.0f;
  }
  if (bad) atomicOr(err, bad);
  __syncthreads();
  const int el = threadIdx.x / LINES, l = threadIdx.x % LINES;
  const bool active = el < count;
  const float gm1inv = (float)g.gm1inv, ggm1 = (float)(g.gamma * g.gm1inv);
#pragma unroll 1
  for (int dir = 0; dir < D; ++dir) {
    if (active) {
      if constexpr (N >= kRows32FromN)
        volume_direction32_rows<D, N, VF>(dir, sp, sa, el, l, tb, gm1inv, ggm1, fs, nelem,
                                          e0 + el, s_left[el][dir], s_ref[el], s_dc[el][dir]);
      else
        volume_direction32<D, N, VF>(dir, sp, sa, el, l, tb, gm1inv, ggm1, fs, nelem, e0 + el,
                                     s_left[el][dir], s_ref[el], s_dc[el][dir]);
    }
    __syncthreads();
  }
  const double dtv = fz.k ? *fz.dt : 0.0;
  double* const uo = fz.u_out ? fz.u_out : u;
  for (int t = threadIdx.x; t < count * P; t += blockDim.x) {
    const int ell = t / P, node = t % P;
    const int e = e0 + ell;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const float val = sa[ell][v][node];
      const long long i = ((long long)e * NV + v) * P + node;
      if (fz.k) {
        double kk = dtv * f2d(val);
        if (stage_k) kk = fma(fz.a, sk[(ell * NV + v) * P + node], kk);
        fz.k[i] = kk;
        uo[i] = u[i] + fz.b * kk;
      } else {
        du[i] = val;
      }
    }
  }
}

// degrees up to 4: at least four CTAs of (at most) 128 threads per SM, i.e.
// at most 128 registers a thread (no spills); higher degrees keep their lines'
// registers
template <int D, int N, int VF, int EPB>
__global__ void __launch_bounds__(EPB* Shape<D, N>::LINES,
                                  (N <= 4 && EPB * Shape<D, N>::LINES <= 128) ? 4 : 1)
    volume_kernel32(double* u, float* __restrict__ du, const float* __restrict__ fs, Geom g,
                    Tables<float> tb, unsigned* __restrict__ err, StageFuse fz) {
  extern __shared__ __align__(16) unsigned char dg_smem[];
  const int e0 = blockIdx.x * EPB;
  const int left = (int)g.nelem - e0;
  volume_batch32<D, N, VF, EPB>(u, du, fs, g, tb, err, fz, e0, left < EPB ? left : EPB,
                                dg_smem);
}

// F* - f(ref_e) of face node l of element e's right face in direction dir,
// stored in fs[dir][v][e][l]; ref holds the references of every element
template <int D, int N, int dir>
__device__ __forceinline__ void face_flux32(const double* __restrict__ u, float* __restrict__ fs,
                                            const Geom& g, int sf, const float* __restrict__ ref,
                                            const double* __restrict__ refE, int e, int l) {
  using S = Shape<D, N>;
  constexpr int NV = S::NV, P = S::P, NF = S::LINES;
  const int nelem = (int)g.nelem;
  const float gamma = (float)g.gamma, gm1inv = (float)g.gm1inv,
              ggm1 = (float)(g.gamma * g.gm1inv), gm1f = (float)g.gm1;
  constexpr int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  const int er = neighbour32(g, e, dir, +1);
  const int nl = line_node<D, N, dir>(l, N), nr = line_node<D, N, dir>(l, 0);
  double cl[NV], cr[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    cl[v] = u[((long long)e * NV + v) * P + nl];
    cr[v] = u[((long long)er * NV + v) * P + nr];
  }
  float rho0, v0[D], p0;
  load_ref<D>(ref, e, rho0, v0, p0);
  const double E0 = refE[e];
  DNode<D> L, R;
  float dmL[D], dmR[D], dEL, dER;
  delta_node<D>(cl, rho0, v0, E0, gm1f, L, dmL, &dEL);
  delta_node<D>(cr, rho0, v0, E0, gm1f, R, dmR, &dER);
  // jumps u_R - u_L, normal-first, for the dissipative fluxes, from the two
  // traces' deviations from the same reference: [rho] = [drho], [m] = [dm] +
  // v0 [drho], [E] = [dE]. Each deviation is one FP64 difference rounded once
  // to FP32, so traces equal to ~1e-16 (a continuous state) round alike unless
  // an FP32 rounding boundary falls between them, about once in 1e8 face
  // nodes, and then by one FP32 ulp of the deviation.
  float dq[NV];
  dq[0] = R.drho - L.drho;
  dq[1] = fmaf(v0[dir], dq[0], dmR[dir] - dmL[dir]);
  dq[2] = fmaf(v0[t1], dq[0], dmR[t1] - dmL[t1]);
  if (D == 3) dq[D] = fmaf(v0[t2], dq[0], dmR[t2] - dmL[t2]);
  dq[D + 1] = dER - dEL;
  const DRef<D> rf = dir_ref<D>(rho0, v0, p0, dir);
  float f[NV];
  delta_surface_flux<D>(sf, to_normal_first<D>(L, dir), to_normal_first<D>(R, dir), rf, dq,
                        gamma, gm1inv, ggm1, f);
  const long long base = (long long)nelem * NF;
  const long long off = (long long)e * NF + l;
  fs[(long long)(dir * NV + 0) * base + off] = f[0];
  fs[(long long)(dir * NV + 1 + dir) * base + off] = f[1];
  fs[(long long)(dir * NV + 1 + t1) * base + off] = f[2];
  if (D == 3) fs[(long long)(dir * NV + 1 + t2) * base + off] = f[D];
  fs[(long long)(dir * NV + NV - 1) * base + off] = f[NV - 1];
}

template <int D, int N, int dir>
__device__ __forceinline__ void surface_body32(const double* __restrict__ u, float* __restrict__ fs,
                                               const Geom& g, int sf,
                                               const float* __restrict__ ref,
                                               const double* __restrict__ refE) {
  constexpr int NF = Shape<D, N>::LINES;
  const long long total = g.nelem * NF;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    face_flux32<D, N, dir>(u, fs, g, sf, ref, refE, (int)(t / NF), (int)(t % NF));
}

template <int D, int N>
__global__ void surface_kernel32(const double* __restrict__ u, float* __restrict__ fs, Geom g,
                                 int sf, const float* __restrict__ ref,
                                 const double* __restrict__ refE) {
  if (blockIdx.y == 0) surface_body32<D, N, 0>(u, fs, g, sf, ref, refE);
  else if (blockIdx.y == 1) surface_body32<D, N, 1>(u, fs, g, sf, ref, refE);
  else surface_body32<D, N, (D == 3 ? 2 : 1)>(u, fs, g, sf, ref, refE);
}

}  // namespace dg
