// The two kernels of one rhs evaluation (Sec. 2.1 DGSEM, Eq. (1) with s = 0):
//
//  surface_kernel: one thread per face node; evaluates the surface flux F*
//    between the trace u_L (node N of the left element) and u_R (node 0 of
//    the right element) of every interface and stores it in the face buffer
//    fs[dir][v][e_left][l] (l = face-node index, see line_node).
//
//  volume_kernel: one CTA per EPB elements, one thread per element line.
//    Prologue: conserved -> primitive at every node into shared memory.
//    Per direction (a runtime loop; the flux is written with the direction's
//    normal component first, so one code body serves every direction): each
//    thread walks its line's N(N+1)/2 node pairs once, evaluating f#(u_a, u_b)
//    a single time for both nodes, since f# is symmetric and the split-form
//    matrix has a zero diagonal:
//      du_a += Ds[a][b] f#(u_a, u_b),  du_b += Ds[b][a] f#(u_a, u_b).
//    Lifting of the face fluxes at the line ends, du += liftR F*_R (node N)
//    + liftL F*_L (node 0), inside each direction phase. Epilogue: one
//    coalesced store of du, or the fused stage update k <- A k + dt du,
//    u <- u + B k.
//
//  volume_pp_kernel (FP64 meshes under kPairParallelElems elements): one
//    thread per node pair instead of per line; with FACES it also evaluates
//    its elements' face fluxes, so that a whole rhs or stage is one launch.
//
// These templates are instantiated for FP64 meshes; FP32 meshes run the
// perturbation-form kernels of dg_rhs32.cuh.
#pragma once
#include "dg_device.cuh"
#include "dg_f32.cuh"

namespace dg {

__device__ __forceinline__ int elem_index(const Geom& g, int x, int y, int z) {
  return x + g.n[0] * (y + g.n[1] * z);
}

// periodic neighbour of element e at offset s = +-1 in direction dir (32-bit)
__device__ __forceinline__ int neighbour32(const Geom& g, int e, int dir, int s) {
  int x = e % g.n[0];
  const int r = e / g.n[0];
  int y = r % g.n[1];
  int z = r / g.n[1];
  if (dir == 0) x = (x + s + g.n[0]) % g.n[0];
  else if (dir == 1) y = (y + s + g.n[1]) % g.n[1];
  else z = (z + s + g.n[2]) % g.n[2];
  return elem_index(g, x, y, z);
}

// node primitives as seen by one direction, normal component first. The two
// leading slots depend on the volume flux: Ranocha's flux takes s0 = rho/2
// and s1 = sig = (gamma-1) rho / p, since the log mean is homogeneous,
//   p_L p_R / ((gamma-1) ln_mean(rho_L p_R, rho_R p_L)) = 1 / ln_mean(sig_L, sig_R),
// which leaves no product of left and right values inside either log mean;
// the other fluxes take s0 = rho, s1 = p.
template <typename R, int D>
struct LinePrim {
  R s0, s1, hp, vn, hvn;
  R vt[D - 1], hvt[D - 1];
};

template <int VF, typename R>
__device__ __forceinline__ void node_slots(R rho, R p, R gm1, R& s0, R& s1) {
  if (VF == kVRanocha) {
    s0 = half(rho);
    s1 = gm1 * rho * rcp(p);
  } else {
    s0 = rho;
    s1 = p;
  }
}

// Ranocha's EC/KEP flux in normal-first order. hp is p/2 (FP64) or p'/2
// (FP32, then the P_e parts are handled by the caller); an = avg(v_n).
template <typename R, int D, bool MIXED = true>
__device__ __forceinline__ void ranocha_nf(const LinePrim<R, D>& L, const LinePrim<R, D>& Rt,
                                           R f[D + 2], R& an) {
  const R rho_ln = ln_mean_halves<R, MIXED>(L.s0, Rt.s0);
  R vd = L.hvn * Rt.vn;
#pragma unroll
  for (int j = 0; j < D - 1; ++j) vd = fma(L.hvt[j], Rt.vt[j], vd);
  // v_L.v_R / 2 + 1 / ((gamma-1) ln_mean(rho/p))
  const R ee = add_inv_ln_mean<R, MIXED>(L.s1, Rt.s1, vd);
  an = L.hvn + Rt.hvn;
  const R f0 = rho_ln * an;
  f[0] = f0;
  f[1] = fma(f0, an, L.hp + Rt.hp);
#pragma unroll
  for (int j = 0; j < D - 1; ++j) f[2 + j] = f0 * (L.hvt[j] + Rt.hvt[j]);
  f[D + 1] = fma(f0, ee, fma(L.hp, Rt.vn, Rt.hp * L.vn));
}

// the other volume fluxes through the generic (Prim) forms, normal first
template <int VF, typename R, int D>
__device__ __forceinline__ void generic_nf(const LinePrim<R, D>& L, const LinePrim<R, D>& Rt,
                                           R gm1inv, R f[D + 2]) {
  Prim<R, D> a, b;
  a.rho = L.s0;
  a.p = L.s1;
  a.v[0] = L.vn;
  b.rho = Rt.s0;
  b.p = Rt.s1;
  b.v[0] = Rt.vn;
#pragma unroll
  for (int j = 0; j < D - 1; ++j) {
    a.v[1 + j] = L.vt[j];
    b.v[1 + j] = Rt.vt[j];
  }
  volume_flux<VF, R, D, 0>(a, b, gm1inv, f);
}

template <int D, int N, typename R, int VF, int EPB>
__device__ __forceinline__ void volume_direction(int dir, R (*sp)[3 + 2 * D][Shape<D, N>::P],
                                                 R (*sa)[D + 2][Shape<D, N>::P], int el, int l,
                                                 const Tables<R>& tb, R gm1inv,
                                                 const R* __restrict__ fs, int nelem, int e,
                                                 int eleft) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, NV = S::NV;
  const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  int node[NP];
  LinePrim<R, D> q[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    node[a] = line_node_rt<D, N>(dir, l, a);
    const int nd = node[a];
    q[a].s0 = sp[el][0][nd];
    q[a].s1 = sp[el][1][nd];
    q[a].hp = sp[el][2][nd];
    q[a].vn = sp[el][3 + dir][nd];
    q[a].hvn = sp[el][3 + D + dir][nd];
    q[a].vt[0] = sp[el][3 + t1][nd];
    q[a].hvt[0] = sp[el][3 + D + t1][nd];
    if (D == 3) {
      q[a].vt[D - 2] = sp[el][3 + t2][nd];
      q[a].hvt[D - 2] = sp[el][3 + D + t2][nd];
    }
  }
  // the line sums continue the total of the earlier directions (the first
  // starts from zero), so that no separate addition of the directions runs
  // (one FP64 addition per node and variable for each direction after the
  // first); the rounding then follows the running total
  int comp[NV];
  comp[0] = 0;
  comp[1] = 1 + dir;
  comp[2] = 1 + t1;
  if (D == 3) comp[D] = 1 + t2;
  comp[D + 1] = D + 1;
  R acc[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[a][v] = dir == 0 ? R(0) : sa[el][comp[v]][node[a]];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
#pragma unroll
    for (int b = a + 1; b < NP; ++b) {
      R f[NV], an = R(0);
      if (VF == kVRanocha) ranocha_nf<R, D>(q[a], q[b], f, an);
      else generic_nf<VF, R, D>(q[a], q[b], gm1inv, f);
      const R dab = tb.Ds[dir][a][b], dba = tb.Ds[dir][b][a];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[a][v] = fma(dab, f[v], acc[a][v]);
        acc[b][v] = fma(dba, f[v], acc[b][v]);
      }
    }
  }
  // lifting at the two ends of the line: + liftR F*_R at node N (this
  // element's face), + liftL F*_L at node 0 (the left neighbour's face); the
  // face-node index of this line is l.
  {
    const R lr = tb.liftR[dir], ll = tb.liftL[dir];
    const long long base = (long long)nelem * Shape<D, N>::LINES;
    const long long oR = (long long)e * Shape<D, N>::LINES + l;
    const long long oL = (long long)eleft * Shape<D, N>::LINES + l;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const long long row = (long long)(dir * NV + comp[c]) * base;
      acc[N][c] = fma(lr, fs[row + oR], acc[N][c]);
      acc[0][c] = fma(ll, fs[row + oL], acc[0][c]);
    }
  }
  // the running totals back to the line's nodes
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int c = 0; c < NV; ++c) sa[el][comp[c]][node[a]] = acc[a][c];
}

// Degrees from kRowsFromN up: the same direction phase with the row node a
// of the pair loop as a loop value. The unrolled body is then one flux per
// partner node b (b > a, a uniform branch) instead of one per pair, a
// quarter of the code at N = 7, and the partner's staged values are read
// from shared memory for each pair instead of being held for the whole line
// (the line-held form needs every register of the thread at N = 7 and
// spills). Row a takes its running total out of the accumulator array,
// continues it over b > a and puts it back, so every node's sum takes its
// terms in the order of volume_direction. The log means take their FP32
// polynomial tails as at the lower degrees (the line-held form at N = 6 and
// 7 ran faster with the shorter code of the FP64 polynomials; the two differ
// by about 1e-16 relative). On GB300 the row loop takes the 3D rhs at N = 7
// from 0.58 to 0.75 G DOF/s and at N = 6 from 0.67 to 0.71; at N = 4 and 5
// the two forms are within 1%.
constexpr int kRowsFromN = 6;

template <int D, int N, typename R, int VF, int EPB>
__device__ __forceinline__ void volume_direction_rows(int dir, R (*sp)[3 + 2 * D][Shape<D, N>::P],
                                                      R (*sa)[D + 2][Shape<D, N>::P], int el,
                                                      int l, const Tables<R>& tb, R gm1inv,
                                                      const R* __restrict__ fs, int nelem, int e,
                                                      int eleft) {
  using S = Shape<D, N>;
  constexpr int NP = S::NP, NV = S::NV;
  const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  const int n0 = line_node_rt<D, N>(dir, l, 0);
  const int ns = line_node_rt<D, N>(dir, l, 1) - n0;  // node stride along the line
  auto stage = [&](int a) {
    const int nd = n0 + a * ns;
    LinePrim<R, D> q;
    q.s0 = sp[el][0][nd];
    q.s1 = sp[el][1][nd];
    q.hp = sp[el][2][nd];
    q.vn = sp[el][3 + dir][nd];
    q.hvn = sp[el][3 + D + dir][nd];
    q.vt[0] = sp[el][3 + t1][nd];
    q.hvt[0] = sp[el][3 + D + t1][nd];
    if (D == 3) {
      q.vt[D - 2] = sp[el][3 + t2][nd];
      q.hvt[D - 2] = sp[el][3 + D + t2][nd];
    }
    return q;
  };
  int comp[NV];
  comp[0] = 0;
  comp[1] = 1 + dir;
  comp[2] = 1 + t1;
  if (D == 3) comp[D] = 1 + t2;
  comp[D + 1] = D + 1;
  R acc[NP][NV];
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[a][v] = dir == 0 ? R(0) : sa[el][comp[v]][n0 + a * ns];
#pragma unroll 1
  for (int a = 0; a < NP - 1; ++a) {
    const LinePrim<R, D> qa = stage(a);
    R ra[NV];
#pragma unroll
    for (int k = 0; k < NP - 1; ++k)
      if (k == a)
#pragma unroll
        for (int v = 0; v < NV; ++v) ra[v] = acc[k][v];
#pragma unroll
    for (int b = 1; b < NP; ++b) {
      if (b > a) {
        const LinePrim<R, D> qb = stage(b);
        R f[NV], an = R(0);
        if (VF == kVRanocha) ranocha_nf<R, D>(qa, qb, f, an);
        else generic_nf<VF, R, D>(qa, qb, gm1inv, f);
        const R dab = tb.Ds[dir][a][b], dba = tb.Ds[dir][b][a];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          ra[v] = fma(dab, f[v], ra[v]);
          acc[b][v] = fma(dba, f[v], acc[b][v]);
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
    const R lr = tb.liftR[dir], ll = tb.liftL[dir];
    const long long base = (long long)nelem * Shape<D, N>::LINES;
    const long long oR = (long long)e * Shape<D, N>::LINES + l;
    const long long oL = (long long)eleft * Shape<D, N>::LINES + l;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      const long long row = (long long)(dir * NV + comp[c]) * base;
      acc[N][c] = fma(lr, fs[row + oR], acc[N][c]);
      acc[0][c] = fma(ll, fs[row + oL], acc[0][c]);
    }
  }
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int c = 0; c < NV; ++c) sa[el][comp[c]][n0 + a * ns] = acc[a][c];
}

// One batch of `count` (<= MAXE) elements from e0: the prologue into shared
// memory (smem: count x (3 + 2D) staged slots, then count x (D + 2)
// accumulators), the D direction phases with one thread per element line,
// and the epilogue. Every thread of the block calls it (it synchronises the
// block); threads beyond count x LINES only help with the prologue and the
// epilogue. In a fused stage (fz.k set) tb holds the coefficients times the
// stage's dt (stage_tables), so that the sums are dt du; otherwise the
// coefficients themselves.
template <int D, int N, typename R, int VF, int MAXE>
__device__ __forceinline__ void volume_batch(double* u, R* __restrict__ du,
                                             const R* __restrict__ fs, const Geom& g,
                                             const Tables<R>& tb, unsigned* __restrict__ err,
                                             const StageFuse& fz, int e0, int count,
                                             unsigned char* smem) {
  using S = Shape<D, N>;
  constexpr int P = S::P, NV = S::NV, LINES = S::LINES;
  constexpr int NC = 3 + 2 * D;  // s0, s1 (see LinePrim), p/2, v[D], v[D]/2
  R(*sp)[NC][P] = reinterpret_cast<R(*)[NC][P]>(smem);
  R(*sa)[NV][P] = reinterpret_cast<R(*)[NV][P]>(smem + sizeof(R) * count * NC * P);
  __shared__ int s_left[MAXE][3];
  const R gm1inv = R(g.gm1inv);
  if ((int)threadIdx.x < count) {
    const int el = threadIdx.x, e = e0 + el;
    const int x = e % g.n[0], r = e / g.n[0], y = r % g.n[1], z = r / g.n[1];
    s_left[el][0] = elem_index(g, x == 0 ? g.n[0] - 1 : x - 1, y, z);
    s_left[el][1] = elem_index(g, x, y == 0 ? g.n[1] - 1 : y - 1, z);
    s_left[el][2] = (D == 3) ? elem_index(g, x, y, z == 0 ? g.n[2] - 1 : z - 1) : 0;
  }
  __syncthreads();
  unsigned bad = 0;
  for (int t = threadIdx.x; t < count * P; t += blockDim.x) {
    const int el = t / P, node = t % P;
    const int e = e0 + el;
    double c[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = u[((long long)e * NV + v) * P + node];
    double rr;
    const Prim<double, D> q = prim_rcp<D>(c, g.gm1, rr);
    bad |= prim_check(q);
    const R p = R(q.p);
    node_slots<VF, R>(R(q.rho), p, R(g.gm1), sp[el][0][node], sp[el][1][node]);
    sp[el][2][node] = half(p);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      sp[el][3 + k][node] = R(q.v[k]);
      sp[el][3 + D + k][node] = half(R(q.v[k]));
    }
  }
  if (bad) atomicOr(err, bad);
  __syncthreads();
  const int el = threadIdx.x / LINES, l = threadIdx.x % LINES;
  const bool active = el < count;
  const int nelem = (int)g.nelem;
#pragma unroll 1
  for (int dir = 0; dir < D; ++dir) {
    if (active) {
      if constexpr (N >= kRowsFromN)
        volume_direction_rows<D, N, R, VF, MAXE>(dir, sp, sa, el, l, tb, gm1inv, fs, nelem,
                                                 e0 + el, s_left[el][dir]);
      else
        volume_direction<D, N, R, VF, MAXE>(dir, sp, sa, el, l, tb, gm1inv, fs, nelem, e0 + el,
                                            s_left[el][dir]);
    }
    __syncthreads();
  }
  // epilogue: the store (or the fused stage update; the sums are dt du)
  double* const uo = fz.u_out ? fz.u_out : u;
  for (int t = threadIdx.x; t < count * P; t += blockDim.x) {
    const int ell = t / P, node = t % P;
    const int e = e0 + ell;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const R val = sa[ell][v][node];
      const long long i = ((long long)e * NV + v) * P + node;
      if (fz.k) {
        // the first stage (A = 0) neither reads k nor lets stale k values in
        double kk = (double)val;
        if (fz.a != 0.0) kk = fma(fz.a, fz.k[i], kk);
        fz.k[i] = kk;
        uo[i] = u[i] + fz.b * kk;
      } else {
        du[i] = val;
      }
    }
  }
}

template <int D, int N, typename R, int VF, int EPB>
__global__ void __launch_bounds__(EPB* Shape<D, N>::LINES)
    volume_kernel(double* u, R* __restrict__ du, const R* __restrict__ fs, Geom g, Tables<R> tb,
                  unsigned* __restrict__ err, StageFuse fz) {
  extern __shared__ __align__(16) unsigned char dg_smem[];
  __shared__ Tables<R> s_tab;  // volume_batch's first barrier follows
  stage_tables<D, N, R>(s_tab, tb, fz.k ? R(*fz.dt) : R(1));
  const int e0 = blockIdx.x * EPB;
  const int left = (int)g.nelem - e0;
  volume_batch<D, N, R, VF, EPB>(u, du, fs, g, s_tab, err, fz, e0, left < EPB ? left : EPB,
                                 dg_smem);
}

// ---- surface ----
// trace state for the surface flux, normal component first; ps is the
// pressure in the additive normal-momentum term (p itself here; the MHD-free
// ensemble kernels pass other offsets); rr = 1/rho
template <typename R, int D>
struct Trace {
  R rho, rr, p, ps, vn, vt[D - 1], mn, mt[D - 1], E;
};

template <typename R, int D>
__device__ __forceinline__ void surface_nf(int sf, const Trace<R, D>& L, const Trace<R, D>& Rt,
                                           R dE, R gamma, R gm1inv, R f[D + 2]) {
  if (sf == kSRanocha) {
    const R rho_ln = ln_mean(L.rho, Rt.rho);
    const R inv = inv_ln_mean(L.rho * Rt.p, Rt.rho * L.p);
    const R an = half(L.vn + Rt.vn);
    const R f0 = rho_ln * an;
    f[0] = f0;
    f[1] = f0 * an + half(L.ps + Rt.ps);
    R vd = L.vn * Rt.vn;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
      f[2 + j] = f0 * half(L.vt[j] + Rt.vt[j]);
      vd += L.vt[j] * Rt.vt[j];
    }
    f[D + 1] = f0 * (half(vd) + L.p * Rt.p * inv * gm1inv) + half(L.p * Rt.vn + Rt.p * L.vn);
    return;
  }
  if (sf == kSChandrashekar) {
    Prim<R, D> a, b;
    a.rho = L.rho;
    a.p = L.p;
    a.v[0] = L.vn;
    b.rho = Rt.rho;
    b.p = Rt.p;
    b.v[0] = Rt.vn;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
      a.v[1 + j] = L.vt[j];
      b.v[1 + j] = Rt.vt[j];
    }
    flux_chandrashekar<R, D, 0>(a, b, gm1inv, f);
    f[1] -= L.p - L.ps;
    return;
  }
  R fl[D + 2], fr[D + 2], dq[D + 2];
  fl[0] = L.mn;
  fr[0] = Rt.mn;
  fl[1] = L.mn * L.vn + L.ps;
  fr[1] = Rt.mn * Rt.vn + Rt.ps;
#pragma unroll
  for (int j = 0; j < D - 1; ++j) {
    fl[2 + j] = L.mn * L.vt[j];
    fr[2 + j] = Rt.mn * Rt.vt[j];
    dq[2 + j] = Rt.mt[j] - L.mt[j];
  }
  fl[D + 1] = (L.E + L.p) * L.vn;
  fr[D + 1] = (Rt.E + Rt.p) * Rt.vn;
  dq[0] = Rt.rho - L.rho;
  dq[1] = Rt.mn - L.mn;
  dq[D + 1] = dE;
  const R c2l = gamma * L.p * L.rr, c2r = gamma * Rt.p * Rt.rr;
  if (sf == kSLLF) {
    // max(c_L, c_R) as the root of max(c_L^2, c_R^2): one square root,
    // within one ulp of the larger sound speed
    const R lam = fmax_nn(fabs(L.vn), fabs(Rt.vn)) + sqrt_pos(fmax_nn(c2l, c2r));
    const R hlam = half(lam);
#pragma unroll
    for (int v = 0; v < D + 2; ++v) f[v] = fma(-hlam, dq[v], half(fl[v] + fr[v]));
    return;
  }
  const R cl = sqrt(c2l), cr = sqrt(c2r);
  const R sL = fmin(L.vn - cl, Rt.vn - cr);
  const R sR = fmax(L.vn + cl, Rt.vn + cr);
#pragma unroll
  for (int v = 0; v < D + 2; ++v) {
    if (sL >= R(0)) f[v] = fl[v];
    else if (sR <= R(0)) f[v] = fr[v];
    else f[v] = (sR * fl[v] - sL * fr[v] + sL * sR * dq[v]) / (sR - sL);
  }
}

// the surface flux of face node l of element e's right face in direction
// dir (the left element e, the right one its +dir neighbour), stored in
// fs[dir][v][e][l]
// a[k] of a D-vector for a runtime k in [0, D)
template <int D>
__device__ __forceinline__ double pick(const double* a, int k) {
  if constexpr (D == 3) return k == 0 ? a[0] : (k == 1 ? a[1] : a[2]);
  else return k == 0 ? a[0] : a[1];
}

// the surface flux of face node l of the right face (direction dir) of
// element e, normal-first: f[0] mass, f[1] normal momentum, f[2..D]
// tangential momenta (directions dir+1, dir+2), f[D+1] energy. dir is a
// value (the face kernel passes a constant, the one-launch small-mesh kernel
// its thread's direction: the same arithmetic either way).
template <int D, int N, typename R>
__device__ __forceinline__ void face_flux_nf_dir(int dir, const double* __restrict__ u,
                                                 const Geom& g, int sf, int e, int l,
                                                 R f[D + 2]) {
  using S = Shape<D, N>;
  constexpr int NV = S::NV, P = S::P;
  const R gamma = R(g.gamma), gm1inv = R(g.gm1inv);
  const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  const int er = neighbour32(g, e, dir, +1);
  const int nl = line_node_rt<D, N>(dir, l, N), nr = line_node_rt<D, N>(dir, l, 0);
  double cl[NV], cr[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    cl[v] = u[((long long)e * NV + v) * P + nl];
    cr[v] = u[((long long)er * NV + v) * P + nr];
  }
  Trace<R, D> L, Rt;
  double rrl, rrr;
  const Prim<double, D> ql = prim_rcp<D>(cl, g.gm1, rrl);
  const Prim<double, D> qr = prim_rcp<D>(cr, g.gm1, rrr);
  L.rr = R(rrl);
  Rt.rr = R(rrr);
  L.rho = R(ql.rho);
  L.p = R(ql.p);
  L.ps = L.p;
  Rt.rho = R(qr.rho);
  Rt.p = R(qr.p);
  Rt.ps = Rt.p;
  // components picked by selects (no indexing of register arrays by a
  // runtime direction)
  L.vn = R(pick<D>(ql.v, dir));
  Rt.vn = R(pick<D>(qr.v, dir));
  L.vt[0] = R(pick<D>(ql.v, t1));
  Rt.vt[0] = R(pick<D>(qr.v, t1));
  if (D == 3) {
    L.vt[D - 2] = R(pick<D>(ql.v, t2));
    Rt.vt[D - 2] = R(pick<D>(qr.v, t2));
  }
  const R dE = R(cr[NV - 1] - cl[NV - 1]);
  L.mn = R(pick<D>(cl + 1, dir));
  Rt.mn = R(pick<D>(cr + 1, dir));
  L.mt[0] = R(pick<D>(cl + 1, t1));
  Rt.mt[0] = R(pick<D>(cr + 1, t1));
  if (D == 3) {
    L.mt[D - 2] = R(pick<D>(cl + 1, t2));
    Rt.mt[D - 2] = R(pick<D>(cr + 1, t2));
  }
  L.E = R(cl[NV - 1]);
  Rt.E = R(cr[NV - 1]);
  surface_nf<R, D>(sf, L, Rt, dE, gamma, gm1inv, f);
}

template <int D, int N, typename R, int dir>
__device__ __forceinline__ void face_flux_nf(const double* __restrict__ u, const Geom& g, int sf,
                                             int e, int l, R f[D + 2]) {
  face_flux_nf_dir<D, N, R>(dir, u, g, sf, e, l, f);
}

template <int D, int N, typename R, int dir>
__device__ __forceinline__ void face_flux(const double* __restrict__ u, R* __restrict__ fs,
                                          const Geom& g, int sf, int e, int l) {
  constexpr int NV = D + 2, NF = Shape<D, N>::LINES;
  constexpr int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  const int nelem = (int)g.nelem;
  R f[NV];
  face_flux_nf<D, N, R, dir>(u, g, sf, e, l, f);
  const long long base = (long long)nelem * NF;
  const long long off = (long long)e * NF + l;
  fs[(long long)(dir * NV + 0) * base + off] = f[0];
  fs[(long long)(dir * NV + 1 + dir) * base + off] = f[1];
  fs[(long long)(dir * NV + 1 + t1) * base + off] = f[2];
  if (D == 3) fs[(long long)(dir * NV + 1 + t2) * base + off] = f[D];
  fs[(long long)(dir * NV + NV - 1) * base + off] = f[NV - 1];
}

// face_flux with the direction as a value: warps whose lanes hold faces of
// different directions run one instruction stream (the same arithmetic)
template <int D, int N, typename R>
__device__ __forceinline__ void face_flux_rt(int dir, const double* __restrict__ u,
                                             R* __restrict__ fs, const Geom& g, int sf, int e,
                                             int l) {
  constexpr int NV = D + 2, NF = Shape<D, N>::LINES;
  const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
  const int nelem = (int)g.nelem;
  R f[NV];
  face_flux_nf_dir<D, N, R>(dir, u, g, sf, e, l, f);
  const long long base = (long long)nelem * NF;
  const long long off = (long long)e * NF + l;
  fs[(long long)(dir * NV + 0) * base + off] = f[0];
  fs[(long long)(dir * NV + 1 + dir) * base + off] = f[1];
  fs[(long long)(dir * NV + 1 + t1) * base + off] = f[2];
  if (D == 3) fs[(long long)(dir * NV + 1 + t2) * base + off] = f[D];
  fs[(long long)(dir * NV + NV - 1) * base + off] = f[NV - 1];
}

template <int D, int N, typename R, int dir>
__device__ __forceinline__ void surface_body(const double* __restrict__ u, R* __restrict__ fs,
                                             const Geom& g, int sf) {
  constexpr int NF = Shape<D, N>::LINES;
  const long long total = g.nelem * NF;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    face_flux<D, N, R, dir>(u, fs, g, sf, (int)(t / NF), (int)(t % NF));
}

template <int D, int N, typename R>
__global__ void surface_kernel(const double* __restrict__ u, R* __restrict__ fs, Geom g, int sf) {
  if (blockIdx.y == 0) surface_body<D, N, R, 0>(u, fs, g, sf);
  else if (blockIdx.y == 1) surface_body<D, N, R, 1>(u, fs, g, sf);
  else surface_body<D, N, R, (D == 3 ? 2 : 1)>(u, fs, g, sf);
}

// ---- pair-parallel volume kernel for tiny meshes (FP64) ----
// One thread per (direction, line, node pair): every pair flux is evaluated
// by its own thread (the line-owning kernel walks a line's N(N+1)/2 pairs in
// one thread; on a mesh of a few hundred elements each SM holds one or two of
// those threads' warps). The fluxes go to shared memory; then one thread per
// (direction, node) sums its pairs in the line-owning kernel's order (the
// other node's index ascending, then the lifting), and the directions are
// added in order, so the result is bitwise that of volume_kernel.
//
// On this GPU a warp's FP64 instruction occupies its sub-partition's FP64
// unit for 64 cycles (half a lane per cycle) whatever its active lanes, so a
// CTA takes EPB elements at once and every phase packs its work items into
// full warps (2D N = 3: two elements per CTA).
//
// With FACES the same launch also evaluates the surface fluxes its elements
// need (both faces in every direction, in shared memory) in warps of their
// own that run beside the prologue and the first pair phase: a whole rhs, or
// a whole Runge-Kutta stage that writes its new state to another buffer
// (neighbours read the input state), in one launch. Each face is then
// evaluated by both of its elements, with the face kernel's arithmetic, so the
// result is the same as with the face kernel.
//
// G: directions per phase (0: all of them when one element's pair fluxes fit
// in 96 KB, else one); EPB: elements per CTA.
template <int D, int N, int G = 0, int EPB = 1>
struct PairPar {
  static constexpr int NP = N + 1, P = Shape<D, N>::P, LINES = Shape<D, N>::LINES,
                       NV = D + 2, NC = 3 + 2 * D;
  static constexpr int NPAIRS = N * (N + 1) / 2;
  static constexpr bool ALLDIRS = D * LINES * NPAIRS * NV * 8 <= 98304;
  static constexpr int GROUP = G > 0 ? G : (ALLDIRS ? D : 1);
  static constexpr int WORK = GROUP * LINES * NPAIRS;  // pair items per element and phase
  // volume threads: the pair items of the CTA's elements, at most 512
  static constexpr int THREADS = EPB * WORK < 512 ? ((EPB * WORK + 31) / 32) * 32 : 512;
  static constexpr int ELEM_SMEM = (NC + NV + GROUP * NV) * P * 8 + WORK * NV * 8;
  static constexpr int SMEM = EPB * ELEM_SMEM;
  // FACES: face warps after the volume threads, one thread per face node of
  // the elements' 2 D faces
  static constexpr int FITEMS = EPB * 2 * D * LINES;
  static constexpr int THREADS_F = THREADS + ((FITEMS + 31) / 32) * 32;
  static_assert(THREADS_F <= 1024, "face warps do not fit the CTA");
  static constexpr int SMEM_F = SMEM + EPB * 2 * D * NV * LINES * 8;
};

// elements per CTA of the one-launch kernel: enough to fill a warp with the
// face nodes of the elements (at most 4)
template <int D, int N>
constexpr int pp_epb() {
  constexpr int per = 2 * D * Shape<D, N>::LINES;
  return per >= 32 ? 1 : (32 / per > 4 ? 4 : 32 / per);
}

// the normal-first component of variable v in direction dir: 0 mass, 1 the
// normal momentum, 2 .. D the momenta of directions dir+1, dir+2, D+1 energy
template <int D>
__device__ __forceinline__ int nf_component(int v, int dir) {
  if (v == 0 || v == D + 1) return v;
  const int k = v - 1;
  return k == dir ? 1 : (k == (dir + 1) % D ? 2 : D);
}

template <int N>
__device__ __forceinline__ void pp_pair_of(int p, int& a, int& b) {
  a = 0;
  while (p >= N - a) {
    p -= N - a;
    ++a;
  }
  b = a + 1 + p;
}

template <int N>
__device__ __forceinline__ int pp_pair_index(int a, int b) {  // a < b
  return a * N - a * (a - 1) / 2 + (b - a - 1);
}

// line l and position i of a node along direction dir (inverse of line_node)
template <int D, int N>
__device__ __forceinline__ void pp_line_of(int dir, int node, int& l, int& i) {
  constexpr int NP = N + 1;
  if (dir == 0) {
    l = node / NP;
    i = node % NP;
  } else if (dir == 1) {
    i = (node / NP) % NP;
    l = (D == 2) ? node % NP : node % NP + NP * (node / (NP * NP));
  } else {
    i = node / (NP * NP);
    l = node % (NP * NP);
  }
}

// The body for the `count` (<= EPB) elements from e0 (every thread of the
// block calls it; it ends with a barrier after its last shared-memory read,
// so a block may run it for one batch after another). smem: C::SMEM bytes
// (C::SMEM_F with FACES).
template <int D, int N, int VF, bool FACES, int G, int EPB, bool CHAIN = false>
__device__ __forceinline__ void pp_elements(double* u, double* __restrict__ du,
                                            const double* __restrict__ fs, const Geom& g,
                                            const Tables<double>& tb, unsigned* __restrict__ err,
                                            const StageFuse& fz, int sfk, int e0, int count,
                                            unsigned char* dg_smem) {
  using C = PairPar<D, N, G, EPB>;
  constexpr int NP = C::NP, P = C::P, NV = C::NV, NC = C::NC, LINES = C::LINES,
                NPAIRS = C::NPAIRS, GROUP = C::GROUP, WORK = C::WORK;
  // per element el: slots sp[NC][P], accumulators sa[NV][P], direction
  // parts sd[GROUP][NV][P] (unless CHAIN), pair fluxes sf[WORK][NV]; FACES: sfc[el] =
  // [side][dir][c][l], side 0 the element's right face, 1 its left face, c in
  // normal-first order
  auto sp = [&](int el) {
    return reinterpret_cast<double(*)[P]>(dg_smem + el * C::ELEM_SMEM);
  };
  auto sa = [&](int el) {
    return reinterpret_cast<double(*)[P]>(dg_smem + el * C::ELEM_SMEM + 8 * NC * P);
  };
  auto sd = [&](int el) {
    return reinterpret_cast<double(*)[NV][P]>(dg_smem + el * C::ELEM_SMEM + 8 * (NC + NV) * P);
  };
  auto sf = [&](int el) {
    return reinterpret_cast<double*>(dg_smem + el * C::ELEM_SMEM +
                                     8 * (NC + NV + GROUP * NV) * P);
  };
  double* sfc = reinterpret_cast<double*>(dg_smem + C::SMEM);
  const int nelem = (int)g.nelem;
  __shared__ int s_left[EPB][3];
  for (int t = threadIdx.x; t < EPB * D; t += blockDim.x)
    s_left[t / D][t % D] = t / D < count ? neighbour32(g, e0 + t / D, t % D, -1) : 0;

  // FACES: the first THREADS threads (the volume threads) do the prologue and
  // the first pair phase, synchronised among themselves by barrier 1, while
  // the face warps evaluate the surface fluxes; all meet at the barrier
  // before the first line sums
  const int wt = FACES ? C::THREADS : (int)blockDim.x;
  if (FACES && (int)threadIdx.x >= C::THREADS) {
    constexpr int PER = 2 * D * LINES;  // face nodes per element
    for (int t = (int)threadIdx.x - C::THREADS; t < C::FITEMS;
         t += (int)blockDim.x - C::THREADS) {
      const int el = t / PER, r = t % PER;
      if (el < count) {
        const int side = r / (D * LINES), dir = (r / LINES) % D, l = r % LINES;
        const int e = e0 + el;
        const int owner = side == 0 ? e : neighbour32(g, e, dir, -1);
        double f[NV];
        face_flux_nf_dir<D, N, double>(dir, u, g, sfk, owner, l, f);
        double* dst = sfc + (long long)el * PER * NV + (side * D + dir) * NV * LINES + l;
#pragma unroll
        for (int c = 0; c < NV; ++c) dst[c * LINES] = f[c];
      }
    }
  }
  unsigned bad = 0;
  for (int t = threadIdx.x; t < EPB * P && (int)threadIdx.x < wt; t += wt) {
    const int el = t / P, node = t % P;
    if (el >= count) continue;
    const int e = e0 + el;
    double c[NV], rr;
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = u[((long long)e * NV + v) * P + node];
    const Prim<double, D> q = prim_rcp<D>(c, g.gm1, rr);
    bad |= prim_check(q);
    double(*spe)[P] = sp(el);
    node_slots<VF, double>(q.rho, q.p, g.gm1, spe[0][node], spe[1][node]);
    spe[2][node] = half(q.p);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      spe[3 + k][node] = q.v[k];
      spe[3 + D + k][node] = half(q.v[k]);
    }
  }
  if (bad) atomicOr(err, bad);
  if (FACES) {
    if ((int)threadIdx.x < C::THREADS) asm volatile("bar.sync 1, %0;" ::"r"(C::THREADS) : "memory");
  } else {
    __syncthreads();
  }
  const long long base = (long long)nelem * LINES;
  const double gm1inv = g.gm1inv;
#pragma unroll 1
  for (int d0 = 0; d0 < D; d0 += GROUP) {
    // pair fluxes of the group's directions, normal-first (volume threads)
    for (int t = threadIdx.x; t < EPB * WORK && (int)threadIdx.x < wt; t += wt) {
      const int el = t / WORK, w = t % WORK;
      if (el >= count) continue;
      double(*spe)[P] = sp(el);
      const int dir = d0 + w / (LINES * NPAIRS);
      const int rem = w % (LINES * NPAIRS);
      const int l = rem / NPAIRS;
      int a, b;
      pp_pair_of<N>(rem % NPAIRS, a, b);
      const int na = line_node_rt<D, N>(dir, l, a), nb = line_node_rt<D, N>(dir, l, b);
      const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
      LinePrim<double, D> qa, qb;
      qa.s0 = spe[0][na];
      qa.s1 = spe[1][na];
      qa.hp = spe[2][na];
      qa.vn = spe[3 + dir][na];
      qa.hvn = spe[3 + D + dir][na];
      qa.vt[0] = spe[3 + t1][na];
      qa.hvt[0] = spe[3 + D + t1][na];
      qb.s0 = spe[0][nb];
      qb.s1 = spe[1][nb];
      qb.hp = spe[2][nb];
      qb.vn = spe[3 + dir][nb];
      qb.hvn = spe[3 + D + dir][nb];
      qb.vt[0] = spe[3 + t1][nb];
      qb.hvt[0] = spe[3 + D + t1][nb];
      if (D == 3) {
        qa.vt[D - 2] = spe[3 + t2][na];
        qa.hvt[D - 2] = spe[3 + D + t2][na];
        qb.vt[D - 2] = spe[3 + t2][nb];
        qb.hvt[D - 2] = spe[3 + D + t2][nb];
      }
      double f[NV], an = 0.0;
      if (VF == kVRanocha) ranocha_nf<double, D>(qa, qb, f, an);
      else generic_nf<VF, double, D>(qa, qb, gm1inv, f);
      double* sfe = sf(el);
#pragma unroll
      for (int v = 0; v < NV; ++v) sfe[w * NV + v] = f[v];
    }
    __syncthreads();
    if constexpr (CHAIN) {
      // CHAIN: per (element, variable, node), the line sums of the group's
      // directions in the line-owning kernel's order, each continuing the
      // running total of the earlier directions, with the lifting at the line
      // ends (face values in normal-first order)
      for (int t = threadIdx.x; t < EPB * NV * P; t += blockDim.x) {
        const int el = t / (NV * P), r = t % (NV * P);
        if (el >= count) continue;
        const int v = r / P, node = r % P;
        const int e = e0 + el;
        const double* sfe = sf(el);
        const double* fce = sfc + (long long)el * 2 * D * LINES * NV;
        double acc = d0 == 0 ? 0.0 : sa(el)[v][node];
        for (int gd = 0; gd < GROUP; ++gd) {
          const int dir = d0 + gd, c = nf_component<D>(v, dir);
          int l, i;
          pp_line_of<D, N>(dir, node, l, i);
          for (int j = 0; j < NP; ++j) {
            if (j == i) continue;
            const int p = j < i ? pp_pair_index<N>(j, i) : pp_pair_index<N>(i, j);
            acc = fma(tb.Ds[dir][i][j], sfe[((gd * LINES + l) * NPAIRS + p) * NV + c], acc);
          }
          if (i == N)
            acc = fma(tb.liftR[dir],
                      FACES ? fce[((0 * D + dir) * NV + c) * LINES + l]
                            : fs[(long long)(dir * NV + v) * base + (long long)e * LINES + l],
                      acc);
          if (i == 0)
            acc = fma(tb.liftL[dir],
                      FACES ? fce[((1 * D + dir) * NV + c) * LINES + l]
                            : fs[(long long)(dir * NV + v) * base +
                                 (long long)s_left[el][dir] * LINES + l],
                      acc);
        }
        sa(el)[v][node] = acc;
      }
      __syncthreads();
    } else {
      // otherwise per (element, direction, node): the line sum on its own
      // (in the same order of pairs), then the lifting (normal-first
      // components back to variables); a direction whose terms cancel exactly
      // keeps its exact zero
      for (int t = threadIdx.x; t < EPB * GROUP * P; t += blockDim.x) {
        const int el = t / (GROUP * P), r = t % (GROUP * P);
        if (el >= count) continue;
        const int gd = r / P, node = r % P, dir = d0 + gd;
        const int e = e0 + el;
        const int t1 = (dir + 1) % D, t2 = (dir + 2) % D;
        int l, i;
        pp_line_of<D, N>(dir, node, l, i);
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0.0;
        const double* sfe = sf(el);
        for (int j = 0; j < NP; ++j) {
          if (j == i) continue;
          const int p = j < i ? pp_pair_index<N>(j, i) : pp_pair_index<N>(i, j);
          const double dij = tb.Ds[dir][i][j];
          const double* fp = sfe + ((gd * LINES + l) * NPAIRS + p) * NV;
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[v] = fma(dij, fp[v], acc[v]);
        }
        int comp[NV];
        comp[0] = 0;
        comp[1] = 1 + dir;
        comp[2] = 1 + t1;
        if (D == 3) comp[D] = 1 + t2;
        comp[D + 1] = D + 1;
        const double* fce = sfc + (long long)el * 2 * D * LINES * NV;
        if (i == N) {
#pragma unroll
          for (int c = 0; c < NV; ++c)
            acc[c] = fma(tb.liftR[dir],
                         FACES ? fce[((0 * D + dir) * NV + c) * LINES + l]
                               : fs[(long long)(dir * NV + comp[c]) * base + (long long)e * LINES + l],
                         acc[c]);
        }
        if (i == 0) {
#pragma unroll
          for (int c = 0; c < NV; ++c)
            acc[c] = fma(tb.liftL[dir],
                         FACES ? fce[((1 * D + dir) * NV + c) * LINES + l]
                               : fs[(long long)(dir * NV + comp[c]) * base +
                                    (long long)s_left[el][dir] * LINES + l],
                         acc[c]);
        }
        double(*sde)[NV][P] = sd(el);
#pragma unroll
        for (int c = 0; c < NV; ++c) sde[gd][comp[c]][node] = acc[c];
      }
      __syncthreads();
      // the directions' sums added in order
      for (int t = threadIdx.x; t < EPB * NV * P; t += blockDim.x) {
        const int el = t / (NV * P), r = t % (NV * P);
        if (el >= count) continue;
        const int v = r / P, node = r % P;
        // the first direction's part starts the sum
        double acc = d0 == 0 ? sd(el)[0][v][node] : sa(el)[v][node] + sd(el)[0][v][node];
#pragma unroll
        for (int gd = 1; gd < GROUP; ++gd) acc += sd(el)[gd][v][node];
        sa(el)[v][node] = acc;
      }
      __syncthreads();
    }
  }
  // epilogue: the CTA's elements are contiguous in the state
  // (CHAIN: tb holds the coefficients times dt, as volume_batch's does, so
  // the sums are already dt du)
  const double dtv = fz.k ? (CHAIN ? 1.0 : *fz.dt) : 0.0;
  double* const uo = fz.u_out ? fz.u_out : u;
  for (int t = threadIdx.x; t < count * NV * P; t += blockDim.x) {
    const int el = t / (NV * P), r = t % (NV * P);
    const int v = r / P, node = r % P;
    const double val = sa(el)[v][node];
    const long long i = (long long)e0 * NV * P + t;
    if (fz.k) {
      double kk = CHAIN ? val : dtv * val;
      if (fz.a != 0.0) kk = fma(fz.a, fz.k[i], kk);
      fz.k[i] = kk;
      uo[i] = u[i] + fz.b * kk;
    } else {
      du[i] = val;
    }
  }
  __syncthreads();
}

template <int D, int N, int VF, bool FACES, int EPB>
__global__ void __launch_bounds__(FACES ? PairPar<D, N, 0, EPB>::THREADS_F
                                        : PairPar<D, N, 0, EPB>::THREADS)
    volume_pp_kernel(double* u, double* __restrict__ du, const double* __restrict__ fs, Geom g,
                     Tables<double> tb, unsigned* __restrict__ err, StageFuse fz, int sfk) {
  extern __shared__ __align__(16) unsigned char dg_smem[];
  const int e0 = blockIdx.x * EPB;
  const int left = (int)g.nelem - e0;
  pp_elements<D, N, VF, FACES, 0, EPB>(u, du, fs, g, tb, err, fz, sfk, e0,
                                       left < EPB ? left : EPB, dg_smem);
}

}  // namespace dg
#include "dg_rhs32.cuh"
namespace dg {

// elements per CTA: about 128 threads, dynamic shared memory <= 96 KB
template <int D, int N, typename R>
struct Launch {
  static constexpr int LINES = Shape<D, N>::LINES;
  static constexpr int BY_THREADS = (128 / LINES) > 0 ? (128 / LINES) : 1;
  static constexpr int PER_ELEM = (3 + 2 * D + D + 2) * Shape<D, N>::P * (int)sizeof(R);
  static constexpr int BY_SMEM = (98304 / PER_ELEM) > 0 ? (98304 / PER_ELEM) : 1;
  static constexpr int EPB = BY_THREADS < BY_SMEM ? BY_THREADS : BY_SMEM;
  static constexpr int SMEM = EPB * PER_ELEM;
};

template <typename K>
cudaError_t allow_smem(K kernel, int bytes) {
  // the 48 KB default covers static and dynamic shared memory together
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  if (bytes + (int)fa.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// the largest shared-memory carveout (the kernel keeps its working set in
// shared memory and streams the rest)
template <typename K>
cudaError_t prefer_shared(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// parts: bit 0 = surface kernel, bit 1 = volume kernel (both for an rhs)
template <int D, int N, typename R, int EPB>
cudaError_t launch_volume_epb(const double* u, R* du, R* fs, const Geom& g, const Tables<R>& tb,
                              int vf, unsigned* err, cudaStream_t st, const StageFuse& fz) {
  using L = Launch<D, N, R>;
  const long long grid = (g.nelem + EPB - 1) / EPB;
  const int threads = EPB * L::LINES;
  constexpr int SM = EPB * L::PER_ELEM;
  cudaError_t e;
  if (vf == kVRanocha) {
    if ((e = allow_smem(volume_kernel<D, N, R, kVRanocha, EPB>, SM)) != cudaSuccess) return e;
    volume_kernel<D, N, R, kVRanocha, EPB><<<(unsigned)grid, threads, SM, st>>>(
        const_cast<double*>(u), du, fs, g, tb, err, fz);
  } else if (vf == kVChandrashekar) {
    if ((e = allow_smem(volume_kernel<D, N, R, kVChandrashekar, EPB>, SM)) != cudaSuccess) return e;
    volume_kernel<D, N, R, kVChandrashekar, EPB><<<(unsigned)grid, threads, SM, st>>>(
        const_cast<double*>(u), du, fs, g, tb, err, fz);
  } else {
    if ((e = allow_smem(volume_kernel<D, N, R, kVCentral, EPB>, SM)) != cudaSuccess) return e;
    volume_kernel<D, N, R, kVCentral, EPB><<<(unsigned)grid, threads, SM, st>>>(
        const_cast<double*>(u), du, fs, g, tb, err, fz);
  }
  return cudaGetLastError();
}

// meshes of fewer elements than this run the pair-parallel FP64 volume kernel
template <int D, int N, int VF, bool FACES>
cudaError_t launch_volume_pp_vf(const double* u, double* du, double* fs, const Geom& g,
                                const Tables<double>& tb, int sf, unsigned* err, cudaStream_t st,
                                const StageFuse& fz) {
  constexpr int EPB = FACES ? pp_epb<D, N>() : 1;
  using C = PairPar<D, N, 0, EPB>;
  constexpr int threads = FACES ? C::THREADS_F : C::THREADS;
  constexpr int smem = FACES ? C::SMEM_F : C::SMEM;
  cudaError_t e;
  if ((e = allow_smem(volume_pp_kernel<D, N, VF, FACES, EPB>, smem)) != cudaSuccess) return e;
  const unsigned grid = (unsigned)((g.nelem + EPB - 1) / EPB);
  volume_pp_kernel<D, N, VF, FACES, EPB><<<grid, threads, smem, st>>>(
      const_cast<double*>(u), du, fs, g, tb, err, fz, sf);
  return cudaGetLastError();
}

// faces: the surface fluxes in the same launch (a whole rhs, or a stage whose
// output buffer is not its input)
template <int D, int N>
cudaError_t launch_volume_pp(const double* u, double* du, double* fs, const Geom& g,
                             const Tables<double>& tb, int vf, int sf, unsigned* err,
                             cudaStream_t st, const StageFuse& fz, bool faces) {
  if (faces) {
    if (vf == kVRanocha)
      return launch_volume_pp_vf<D, N, kVRanocha, true>(u, du, fs, g, tb, sf, err, st, fz);
    if (vf == kVChandrashekar)
      return launch_volume_pp_vf<D, N, kVChandrashekar, true>(u, du, fs, g, tb, sf, err, st, fz);
    return launch_volume_pp_vf<D, N, kVCentral, true>(u, du, fs, g, tb, sf, err, st, fz);
  }
  if (vf == kVRanocha)
    return launch_volume_pp_vf<D, N, kVRanocha, false>(u, du, fs, g, tb, sf, err, st, fz);
  if (vf == kVChandrashekar)
    return launch_volume_pp_vf<D, N, kVChandrashekar, false>(u, du, fs, g, tb, sf, err, st, fz);
  return launch_volume_pp_vf<D, N, kVCentral, false>(u, du, fs, g, tb, sf, err, st, fz);
}

// FP32 kernels: elements per CTA as for FP64 (about 128 threads, dynamic
// shared memory <= 96 KB)
template <int D, int N>
struct Launch32 {
  static constexpr int LINES = Shape<D, N>::LINES;
  static constexpr int BY_THREADS = (128 / LINES) > 0 ? (128 / LINES) : 1;
  // staged slots and accumulators (FP32) and the staged RK register (FP64)
  static constexpr int PER_ELEM = volume32_smem<D, N>(1);
  static constexpr int BY_SMEM = (98304 / PER_ELEM) > 0 ? (98304 / PER_ELEM) : 1;
  static constexpr int EPB = BY_THREADS < BY_SMEM ? BY_THREADS : BY_SMEM;
};

template <int D, int N, int EPB>
cudaError_t launch_volume32_epb(const double* u, float* du, float* fs, const Geom& g,
                                const Tables<float>& tb, int vf, unsigned* err, cudaStream_t st,
                                const StageFuse& fz) {
  using L = Launch32<D, N>;
  const long long grid = (g.nelem + EPB - 1) / EPB;
  const int threads = EPB * L::LINES;
  constexpr int SM = volume32_smem<D, N>(EPB);
  cudaError_t e;
  if (vf == kVRanocha) {
    if ((e = allow_smem(volume_kernel32<D, N, kVRanocha, EPB>, SM)) != cudaSuccess ||
        (e = prefer_shared(volume_kernel32<D, N, kVRanocha, EPB>)) != cudaSuccess)
      return e;
    volume_kernel32<D, N, kVRanocha, EPB><<<(unsigned)grid, threads, SM, st>>>(
        const_cast<double*>(u), du, fs, g, tb, err, fz);
  } else if (vf == kVChandrashekar) {
    if ((e = allow_smem(volume_kernel32<D, N, kVChandrashekar, EPB>, SM)) != cudaSuccess ||
        (e = prefer_shared(volume_kernel32<D, N, kVChandrashekar, EPB>)) != cudaSuccess)
      return e;
    volume_kernel32<D, N, kVChandrashekar, EPB><<<(unsigned)grid, threads, SM, st>>>(
        const_cast<double*>(u), du, fs, g, tb, err, fz);
  } else {
    if ((e = allow_smem(volume_kernel32<D, N, kVCentral, EPB>, SM)) != cudaSuccess ||
        (e = prefer_shared(volume_kernel32<D, N, kVCentral, EPB>)) != cudaSuccess)
      return e;
    volume_kernel32<D, N, kVCentral, EPB><<<(unsigned)grid, threads, SM, st>>>(
        const_cast<double*>(u), du, fs, g, tb, err, fz);
  }
  return cudaGetLastError();
}

// FP64 meshes under kPairParallelElems elements run a whole rhs (parts = 3),
// or a stage whose output buffer is not its input, as one launch of the
// pair-parallel kernel with its face fluxes; the separate parts stay
// available. Other meshes with fewer elements than about two CTAs per SM run
// one element per CTA (and the face kernel in 64-thread blocks), spreading
// the FP64 work (2 lanes per clock per SM) over more SMs; the arithmetic per
// node, and so the result, is the same. FP32 meshes first write the
// per-element references (part 1), which both flux kernels read.
template <int D, int N, typename R>
cudaError_t launch_rhs_dn(const double* u, R* du, R* fs, const Geom& g, const Tables<R>& tb,
                          int vf, int sf, unsigned* err, cudaStream_t st, int parts,
                          const StageFuse& fz) {
  constexpr bool F32 = sizeof(R) == 4;
  if constexpr (!F32) {
    // small FP64 meshes: the whole rhs (or a stage into another buffer) in
    // one launch
    if (parts == 3 && g.nelem < kPairParallelElems && (!fz.k || (fz.u_out && fz.u_out != u)))
      return launch_volume_pp<D, N>(u, du, fs, g, tb, vf, sf, err, st, fz, true);
  }
  if (parts & 1) {
    const long long total = g.nelem * Shape<D, N>::LINES;
    const int threads = (total < 152LL * 4 * 256) ? 64 : 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if constexpr (F32) {
      if (!fz.ref || !fz.refE) return cudaErrorInvalidValue;
      long long eb = (g.nelem + 127) / 128;
      if (eb > 152 * 16) eb = 152 * 16;
      ref_kernel<D><<<(unsigned)eb, 128, 0, st>>>(u, fz.ref, fz.refE, g.nelem, N + 1, g.gm1,
                                                  g.gm1inv);
      surface_kernel32<D, N><<<dim3((unsigned)blocks, D), threads, 0, st>>>(u, fs, g, sf, fz.ref,
                                                                            fz.refE);
    } else {
      surface_kernel<D, N, R><<<dim3((unsigned)blocks, D), threads, 0, st>>>(u, fs, g, sf);
    }
  }
  if (!(parts & 2)) return cudaGetLastError();
  if constexpr (F32) {
    if (!fz.ref || !fz.refE) return cudaErrorInvalidValue;
    constexpr int EPB = Launch32<D, N>::EPB;
    if (EPB > 1 && g.nelem < 2LL * 152 * EPB)
      return launch_volume32_epb<D, N, 1>(u, du, fs, g, tb, vf, err, st, fz);
    return launch_volume32_epb<D, N, EPB>(u, du, fs, g, tb, vf, err, st, fz);
  } else {
    using L = Launch<D, N, R>;
    constexpr int EPB = L::EPB;
    if (g.nelem < kPairParallelElems)
      return launch_volume_pp<D, N>(u, du, fs, g, tb, vf, sf, err, st, fz, false);
    if (EPB > 1 && g.nelem < 2LL * 152 * EPB)
      return launch_volume_epb<D, N, R, 1>(u, du, fs, g, tb, vf, err, st, fz);
    return launch_volume_epb<D, N, R, EPB>(u, du, fs, g, tb, vf, err, st, fz);
  }
}

template <int D, typename R>
cudaError_t launch_rhs_d(int N, const double* u, R* du, R* fs, const Geom& g, const Tables<R>& tb,
                         int vf, int sf, unsigned* err, cudaStream_t st, int parts,
                         const StageFuse& fz) {
  switch (N) {
    case 1: return launch_rhs_dn<D, 1, R>(u, du, fs, g, tb, vf, sf, err, st, parts, fz);
    case 2: return launch_rhs_dn<D, 2, R>(u, du, fs, g, tb, vf, sf, err, st, parts, fz);
    case 3: return launch_rhs_dn<D, 3, R>(u, du, fs, g, tb, vf, sf, err, st, parts, fz);
    case 4: return launch_rhs_dn<D, 4, R>(u, du, fs, g, tb, vf, sf, err, st, parts, fz);
    case 5: return launch_rhs_dn<D, 5, R>(u, du, fs, g, tb, vf, sf, err, st, parts, fz);
    case 6: return launch_rhs_dn<D, 6, R>(u, du, fs, g, tb, vf, sf, err, st, parts, fz);
    case 7: return launch_rhs_dn<D, 7, R>(u, du, fs, g, tb, vf, sf, err, st, parts, fz);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
