// 3D ideal magnetohydrodynamics (MHD) on the uniform periodic Cartesian mesh
// with the Powell non-conservative term: the paper's two MHD solvers for the
// Alfven-wave runs of Sec. 3.1, the weak-form DGSEM (the split form with the
// central volume flux, written in its strong form) with HLL or local
// Lax-Friedrichs faces, and flux differencing with an entropy-conservative
// (EC) two-point flux in the volume and at the faces.
//
// Variables u = (rho, rho v, E, B), E = p/(gamma-1) + rho|v|^2/2 + |B|^2/2.
// Weak form: with D the LGL derivative matrix, Dn = -(2/h) D, liftR =
// -(2/h)/w_N and liftL = +(2/h)/w_0 per direction, node i of a line gets
//   du_i += sum_b Dn_ib f(u_b) + [i = N] liftR (F*_R - f(u_i))
//                              + [i = 0] liftL (F*_L - f(u_i)),
// which equals -(2/h) (sum_m Dt_im (f_i + f_m)/2 + [i = N] F*_R/w_N -
// [i = 0] F*_L/w_0), Dt = 2D - W^-1 B, since the rows of Dt sum to -B_ii/w_i.
// EC flux differencing: the split form itself, -(2/h) (sum_m Dt_im
// f#(u_i, u_m) + the same lifting of F*), f# the EC flux.
// The Powell term is -Phi(u_i) div B_i with Phi = (0, B, v.B, v) and div B
// the split-form derivative of B_n (central two-point value (B_i + B_m)/2,
// the interface average {B_n} at faces): the kernels accumulate -div B and
// add Phi times it.
//
// Kernels of one rhs evaluation:
//   mhd_surface_kernel: one thread per face node; F* = LLF(u_L, u_R) with
//     lambda = max(|v_n,L|, |v_n,R|) + max(c_f,L, c_f,R), HLL with S_L =
//     min(v_n,L - c_f,L, v_n,R - c_f,R), S_R = max(v_n,L + c_f,L, v_n,R +
//     c_f,R), or the EC flux; and {B_n}; nine values per face node in
//     fs[dir][q][e_left][l].
//   mhd_volume_kernel (weak form): one CTA per EPB elements, one thread per
//     node; per direction each thread writes f(u_i) (B_n in the slot of the
//     zero normal induction flux) to shared memory, then applies its line's
//     row of Dn and the lifting; epilogue: the Powell term, then the store
//     of du or the fused stage update.
//   mhd_volume_ec_kernel (EC flux differencing): one element per CTA; per
//     direction one thread per (line, node pair) evaluates f# once for both
//     nodes, then one thread per node sums its line (below).
//   mhd_speed_kernel: one warp per element; sum_dir (2/h) max(|v_dir| + c_f)
//     into the mesh's wave-speed word (CFL step).
#include <cuda_runtime.h>

#include "dg_curved.cuh"  // pair_of, pair_index, line_of
#include "dg_device.cuh"
#include "dg_mhd_decl.cuh"

namespace dg {

namespace {

constexpr int kMV = 8;  // conserved MHD variables
constexpr int kMQ = 9;  // face values: F* (8) and {B_n}
constexpr int kMhdLlf = 0, kMhdHll = 1, kMhdEc = 2;  // surface fluxes
// volume CTAs of about kMhdThreads threads; those up to that size ask for
// kMhdMinBlocks resident CTAs per SM (80 registers a thread at 256 threads)
constexpr int kMhdThreads = 256;
constexpr int kMhdMinBlocks = 3;

struct MState {
  double rho, rr, v[3], p, B[3], b2, vb, pt, E;
};

__device__ __forceinline__ MState mhd_state(const double* c, double gm1, unsigned& bad) {
  MState s;
  s.rho = c[0];
  const double rr = 1.0 / c[0];
  s.rr = rr;
  double mv = 0.0, b2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.v[k] = c[1 + k] * rr;
    s.B[k] = c[5 + k];
    mv = fma(c[1 + k], s.v[k], mv);
    b2 = fma(s.B[k], s.B[k], b2);
  }
  s.E = c[4];
  s.b2 = b2;
  s.p = gm1 * (c[4] - 0.5 * mv - 0.5 * b2);
  s.pt = s.p + 0.5 * b2;
  s.vb = s.v[0] * s.B[0] + s.v[1] * s.B[1] + s.v[2] * s.B[2];
  if (!(s.rho > 0.0)) bad |= kErrRho;
  if (!(s.p > 0.0)) bad |= kErrP;
  if (!isfinite(s.rho) || !isfinite(s.p)) bad |= kErrNaN;
  return s;
}

// physical flux in direction DIR (the B_DIR entry is zero)
template <int DIR>
__device__ __forceinline__ void mhd_flux(const MState& s, const double* c, double* f) {
  const double vn = s.v[DIR], bn = s.B[DIR];
  f[0] = c[1 + DIR];
#pragma unroll
  for (int k = 0; k < 3; ++k) f[1 + k] = c[1 + DIR] * s.v[k] - bn * s.B[k];
  f[1 + DIR] += s.pt;
  f[4] = vn * (s.E + s.pt) - bn * s.vb;
#pragma unroll
  for (int k = 0; k < 3; ++k) f[5 + k] = (k == DIR) ? 0.0 : vn * s.B[k] - bn * s.v[k];
}

// square of the fast magnetosonic speed in direction DIR; the discriminant
// is >= (a^2 - b^2)^2 >= 0 in exact arithmetic and is clamped at zero
// against rounding
template <int DIR>
__device__ __forceinline__ double fast_speed2(const MState& s, double gamma) {
  const double a2 = gamma * s.p * s.rr;
  const double b2 = s.b2 * s.rr;
  const double bn2 = s.B[DIR] * s.B[DIR] * s.rr;
  const double q = a2 + b2;
  return 0.5 * (q + sqrt(fmax(q * q - 4.0 * a2 * bn2, 0.0)));
}

// node quantities of the entropy-conservative two-point flux, pre-scaled so
// that each mean is one addition: beta = rho/(2p), hv = v/2, hB = B/2,
// pm = (rho + beta |B|^2)/2, qv2 = |v|^2/4, qB2 = |B|^2/4, hvB = v.B/2
struct ECq {
  double rho, beta, hv[3], hB[3], pm, qv2, qB2, hvB;
};

__device__ __forceinline__ ECq ec_of(const MState& s) {
  ECq q;
  q.rho = s.rho;
  q.beta = 0.5 * s.rho / s.p;
  double v2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q.hv[k] = 0.5 * s.v[k];
    q.hB[k] = 0.5 * s.B[k];
    v2 = fma(s.v[k], s.v[k], v2);
  }
  q.pm = 0.5 * fma(q.beta, s.b2, s.rho);
  q.qv2 = 0.25 * v2;
  q.qB2 = 0.25 * s.b2;
  q.hvB = 0.5 * s.vb;
  return q;
}

// Entropy-conservative two-point flux in direction DIR, the flux that
// satisfies [[w]] . f + {B_n} [[theta]] = [[psi_n]] with the Powell term in
// split form (theta = 2 beta v.B, psi_n = rho v_n + beta v_n |B|^2):
//   f_rho = rho_ln {v_n},  f_m = f_rho {v} - {B_n}{B} + ({rho} + {beta|B|^2})/(2{beta}) e_n,
//   f_B = {v_n}{B} - {B_n}{v} (zero in component DIR),
//   f_E = f_rho (1/(2(gamma-1) beta_ln) - {|v|^2}/2) + f_m.{v} + f_B.{B}
//         - {v_n}{|B|^2}/2 + {B_n}{v.B}.
template <int DIR>
__device__ __forceinline__ void mhd_ec_flux(const ECq& a, const ECq& b, double hgm1inv,
                                            double* f) {
  double va[3], Ba[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    va[k] = a.hv[k] + b.hv[k];
    Ba[k] = a.hB[k] + b.hB[k];
  }
  const double rho_ln = ln_mean(a.rho, b.rho);
  const double inv_beta_ln = inv_ln_mean(a.beta, b.beta);
  const double f0 = rho_ln * va[DIR];
  f[0] = f0;
#pragma unroll
  for (int k = 0; k < 3; ++k) f[1 + k] = fma(f0, va[k], -Ba[DIR] * Ba[k]);
  f[1 + DIR] += (a.pm + b.pm) / (a.beta + b.beta);
#pragma unroll
  for (int k = 0; k < 3; ++k) f[5 + k] = (k == DIR) ? 0.0 : fma(va[DIR], Ba[k], -Ba[DIR] * va[k]);
  double e = f0 * fma(hgm1inv, inv_beta_ln, -(a.qv2 + b.qv2));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    e = fma(f[1 + k], va[k], e);
    if (k != DIR) e = fma(f[5 + k], Ba[k], e);
  }
  e = fma(-va[DIR], a.qB2 + b.qB2, e);
  f[4] = fma(Ba[DIR], a.hvB + b.hvB, e);
}

template <int N, int DIR, int SF>
__device__ __forceinline__ void mhd_surface_body(const double* __restrict__ u,
                                                 double* __restrict__ fs, const Geom& g,
                                                 unsigned& bad) {
  constexpr int NP = N + 1, P = NP * NP * NP, NF = NP * NP;
  const long long total = g.nelem * NF;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / NF;
    const int l = (int)(t % NF);
    const long long er = neighbour(g, e, DIR, +1);
    const int nl = line_node<3, N, DIR>(l, N), nr = line_node<3, N, DIR>(l, 0);
    double cl[kMV], cr[kMV];
#pragma unroll
    for (int v = 0; v < kMV; ++v) {
      cl[v] = u[(e * kMV + v) * P + nl];
      cr[v] = u[(er * kMV + v) * P + nr];
    }
    const MState sl = mhd_state(cl, g.gm1, bad), sr = mhd_state(cr, g.gm1, bad);
    double fl[kMV], fr[kMV];
    mhd_flux<DIR>(sl, cl, fl);
    mhd_flux<DIR>(sr, cr, fr);
    const long long base = g.nelem * NF;
    const long long off = e * NF + l;
    if (SF == kMhdEc) {
      double f[kMV];
      mhd_ec_flux<DIR>(ec_of(sl), ec_of(sr), 0.5 * g.gm1inv, f);
#pragma unroll
      for (int v = 0; v < kMV; ++v) fs[(long long)(DIR * kMQ + v) * base + off] = f[v];
    } else if (SF == kMhdHll) {
      const double cfl = sqrt(fast_speed2<DIR>(sl, g.gamma));
      const double cfr = sqrt(fast_speed2<DIR>(sr, g.gamma));
      const double sL = fmin(sl.v[DIR] - cfl, sr.v[DIR] - cfr);
      const double sR = fmax(sl.v[DIR] + cfl, sr.v[DIR] + cfr);
      const double inv = 1.0 / (sR - sL);
#pragma unroll
      for (int v = 0; v < kMV; ++v) {
        double F;
        if (sL >= 0.0) F = fl[v];
        else if (sR <= 0.0) F = fr[v];
        else F = (sR * fl[v] - sL * fr[v] + sL * sR * (cr[v] - cl[v])) * inv;
        fs[(long long)(DIR * kMQ + v) * base + off] = F;
      }
    } else {
      // max(c_L, c_R) = sqrt(max(c_L^2, c_R^2)) exactly (sqrt is monotone
      // and correctly rounded)
      const double lam = fmax(fabs(sl.v[DIR]), fabs(sr.v[DIR])) +
                         sqrt(fmax(fast_speed2<DIR>(sl, g.gamma), fast_speed2<DIR>(sr, g.gamma)));
#pragma unroll
      for (int v = 0; v < kMV; ++v)
        fs[(long long)(DIR * kMQ + v) * base + off] =
            0.5 * (fl[v] + fr[v]) - 0.5 * lam * (cr[v] - cl[v]);
    }
    fs[(long long)(DIR * kMQ + 8) * base + off] = 0.5 * (cl[5 + DIR] + cr[5 + DIR]);
  }
}

template <int N, int SF>
__global__ void mhd_surface_kernel(const double* __restrict__ u, double* __restrict__ fs, Geom g,
                                   unsigned* __restrict__ err) {
  unsigned bad = 0;
  if (blockIdx.y == 0) mhd_surface_body<N, 0, SF>(u, fs, g, bad);
  else if (blockIdx.y == 1) mhd_surface_body<N, 1, SF>(u, fs, g, bad);
  else mhd_surface_body<N, 2, SF>(u, fs, g, bad);
  if (bad) atomicOr(err, bad);
}

// one direction of the volume pass for the thread's node (index ia along
// DIR). The normal induction flux v_n B_n - B_n v_n is zero, so its shared-
// memory slot 5 + DIR carries B_n instead, whose derivative goes to -div B;
// du of B_n gets only the lifting of F*_{5+DIR} (the LLF dissipation).
// Contributions accumulate straight into acc and divneg.
template <int N, int DIR, int EPB>
__device__ __forceinline__ void mhd_direction(const MState& s, const double* c,
                                              double (*sf)[kMV][(N + 1) * (N + 1) * (N + 1)],
                                              const double (*sD)[N + 1][N + 1], int el, int node,
                                              bool active, long long e, const Geom& g,
                                              const Tables<double>& tb,
                                              const double* __restrict__ fs, double* acc,
                                              double& divneg) {
  constexpr int NP = N + 1, NF = NP * NP;
  constexpr int STRIDE = DIR == 0 ? 1 : (DIR == 1 ? NP : NF);
  constexpr int QB = 5 + DIR;  // the slot of B_n
  if (active) {
    double f[kMV];
    mhd_flux<DIR>(s, c, f);
    f[QB] = s.B[DIR];
#pragma unroll
    for (int q = 0; q < kMV; ++q) sf[el][q][node] = f[q];
  }
  __syncthreads();
  if (active) {
    const int ia = (node / STRIDE) % NP;
    const int first = node - ia * STRIDE;
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      const double w = sD[DIR][ia][b];
#pragma unroll
      for (int q = 0; q < kMV; ++q) {
        if (q == QB) divneg = fma(w, sf[el][q][first + b * STRIDE], divneg);
        else acc[q] = fma(w, sf[el][q][first + b * STRIDE], acc[q]);
      }
    }
    if (ia == N || ia == 0) {
      // face-node index of this line (see line_node)
      const int l = DIR == 0 ? node / NP : (DIR == 1 ? node % NP + NP * (node / NF) : node % NF);
      const long long ef = ia == N ? e : neighbour(g, e, DIR, -1);
      const double lift = ia == N ? tb.liftR[DIR] : tb.liftL[DIR];
      const long long base = g.nelem * NF;
      const double* src = fs + (long long)DIR * kMQ * base + ef * NF + l;
#pragma unroll
      for (int q = 0; q < kMV; ++q) {
        if (q == QB) acc[q] = fma(lift, src[q * base], acc[q]);
        else acc[q] = fma(lift, src[q * base] - sf[el][q][node], acc[q]);
      }
      divneg = fma(lift, src[8 * base] - sf[el][QB][node], divneg);
    }
  }
  __syncthreads();
}

template <int N, int EPB>
__global__ void __launch_bounds__(EPB*(N + 1) * (N + 1) * (N + 1),
                                  (EPB * (N + 1) * (N + 1) * (N + 1) <= kMhdThreads) ? kMhdMinBlocks
                                                                                   : 1)
    mhd_volume_kernel(double* u, double* __restrict__ du, const double* __restrict__ fs, Geom g,
                      Tables<double> tb, int powell, unsigned* __restrict__ err, StageFuse fz) {
  constexpr int NP = N + 1, P = NP * NP * NP;
  extern __shared__ __align__(16) unsigned char dg_smem[];
  double(*sf)[kMV][P] = reinterpret_cast<double(*)[kMV][P]>(dg_smem);
  // the derivative rows, indexed per thread: from shared memory rather than
  // the parameter bank, whose divergent reads serialise
  __shared__ double sD[3][NP][NP];
  for (int t = threadIdx.x; t < 3 * NP * NP; t += blockDim.x)
    sD[t / (NP * NP)][(t / NP) % NP][t % NP] = tb.Ds[t / (NP * NP)][(t / NP) % NP][t % NP];
  const int el = threadIdx.x / P, node = threadIdx.x % P;
  const long long e = (long long)blockIdx.x * EPB + el;
  const bool active = e < g.nelem;
  double c[kMV];
  if (active) {
#pragma unroll
    for (int v = 0; v < kMV; ++v) c[v] = u[(e * kMV + v) * P + node];
  } else {
#pragma unroll
    for (int v = 0; v < kMV; ++v) c[v] = (v == 0 || v == 4) ? 1.0 : 0.0;
  }
  unsigned bad = 0;
  const MState s = mhd_state(c, g.gm1, bad);
  if (bad && active) atomicOr(err, bad);
  double acc[kMV], divneg = 0.0;
#pragma unroll
  for (int v = 0; v < kMV; ++v) acc[v] = 0.0;
  mhd_direction<N, 0, EPB>(s, c, sf, sD, el, node, active, e, g, tb, fs, acc, divneg);
  mhd_direction<N, 1, EPB>(s, c, sf, sD, el, node, active, e, g, tb, fs, acc, divneg);
  mhd_direction<N, 2, EPB>(s, c, sf, sD, el, node, active, e, g, tb, fs, acc, divneg);
  if (!active) return;
  if (powell) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc[1 + k] = fma(s.B[k], divneg, acc[1 + k]);
      acc[5 + k] = fma(s.v[k], divneg, acc[5 + k]);
    }
    acc[4] = fma(s.vb, divneg, acc[4]);
  }
  const double dtv = fz.k ? *fz.dt : 0.0;
  double* const uo = fz.u_out ? fz.u_out : u;
#pragma unroll
  for (int v = 0; v < kMV; ++v) {
    const long long i = (e * kMV + v) * P + node;
    if (fz.k) {
      // the first stage (A = 0) neither reads k nor lets stale k values in
      double kk = dtv * acc[v];
      if (fz.a != 0.0) kk = fma(fz.a, fz.k[i], kk);
      fz.k[i] = kk;
      uo[i] = u[i] + fz.b * kk;
    } else {
      du[i] = acc[v];
    }
  }
}

// ---- entropy-conservative flux differencing: one element per CTA ----
// Per direction, one thread per (line, node pair) evaluates the EC flux once
// for both nodes into shared memory (the flux is symmetric and the split-
// form matrix has a zero diagonal); then one thread per node sums
// Ds_ij f#(u_i, u_j) over its line, the Powell part Ds_ij (B_i + B_j)/2 of
// -div B, and the lifting of F* and {B_n} at the line ends (Ds = -(2/h) Dt,
// the split form of the oracle). Epilogue: the Powell term, the store or the
// fused stage update.
template <int N>
struct MPairs {
  static constexpr int NP = N + 1, P = NP * NP * NP, LINES = NP * NP;
  static constexpr int NPAIRS = N * (N + 1) / 2;
  static constexpr int WORK = LINES * NPAIRS;
  static constexpr int MAXW = WORK > P ? WORK : P;
  static constexpr int THREADS = MAXW < 512 ? ((MAXW + 31) / 32) * 32 : 512;
  static constexpr int NQ = 12;  // the ECq slots: rho, beta, hv, hB, pm, qv2, qB2, hvB
  static constexpr int SMEM = (NQ + kMV + 1) * P * (int)sizeof(double) +
                              WORK * kMV * (int)sizeof(double);
};

template <int N>
__device__ __forceinline__ ECq ec_load(const double (*sq)[(N + 1) * (N + 1) * (N + 1)], int n) {
  ECq q;
  q.rho = sq[0][n];
  q.beta = sq[1][n];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q.hv[k] = sq[2 + k][n];
    q.hB[k] = sq[5 + k][n];
  }
  q.pm = sq[8][n];
  q.qv2 = sq[9][n];
  q.qB2 = sq[10][n];
  q.hvB = sq[11][n];
  return q;
}

template <int N, int DIR>
__device__ __forceinline__ void mhd_ec_direction(const double (*sq)[(N + 1) * (N + 1) * (N + 1)],
                                                 double (*sa)[(N + 1) * (N + 1) * (N + 1)],
                                                 double* pf, const double (*sD)[N + 1][N + 1],
                                                 long long e, const Geom& g,
                                                 const Tables<double>& tb,
                                                 const double* __restrict__ fs) {
  using C = MPairs<N>;
  constexpr int NP = C::NP, P = C::P, LINES = C::LINES, NPAIRS = C::NPAIRS;
  for (int w = threadIdx.x; w < C::WORK; w += blockDim.x) {
    const int l = w / NPAIRS;
    int a, b;
    pair_of<N>(w % NPAIRS, a, b);
    double f[kMV];
    mhd_ec_flux<DIR>(ec_load<N>(sq, line_node<3, N, DIR>(l, a)),
                     ec_load<N>(sq, line_node<3, N, DIR>(l, b)), 0.5 * g.gm1inv, f);
#pragma unroll
    for (int v = 0; v < kMV; ++v) pf[v * C::WORK + w] = f[v];
  }
  __syncthreads();
  for (int node = threadIdx.x; node < P; node += blockDim.x) {
    int l, i;
    line_of<N>(DIR, node, l, i);
    // the line sums continue the running totals of the earlier directions
    double acc[kMV], dn = sa[kMV][node];
#pragma unroll
    for (int v = 0; v < kMV; ++v) acc[v] = sa[v][node];
    const double bi = sq[5 + DIR][node];  // B_n / 2
    for (int j = 0; j < NP; ++j) {
      if (j == i) continue;
      const int p = j < i ? pair_index<N>(j, i) : pair_index<N>(i, j);
      const double dij = sD[DIR][i][j];
#pragma unroll
      for (int v = 0; v < kMV; ++v) acc[v] = fma(dij, pf[v * C::WORK + l * NPAIRS + p], acc[v]);
      dn = fma(dij, bi + sq[5 + DIR][line_node<3, N, DIR>(l, j)], dn);
    }
    if (i == N || i == 0) {
      const long long ef = i == N ? e : neighbour(g, e, DIR, -1);
      const double lift = i == N ? tb.liftR[DIR] : tb.liftL[DIR];
      const long long base = g.nelem * LINES;
      const double* src = fs + (long long)DIR * kMQ * base + ef * LINES + l;
#pragma unroll
      for (int v = 0; v < kMV; ++v) acc[v] = fma(lift, src[v * base], acc[v]);
      dn = fma(lift, src[8 * base], dn);
    }
#pragma unroll
    for (int v = 0; v < kMV; ++v) sa[v][node] = acc[v];
    sa[kMV][node] = dn;
  }
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(MPairs<N>::THREADS)
    mhd_volume_ec_kernel(double* u, double* __restrict__ du, const double* __restrict__ fs, Geom g,
                         Tables<double> tb, int powell, unsigned* __restrict__ err, StageFuse fz) {
  using C = MPairs<N>;
  constexpr int NP = C::NP, P = C::P;
  extern __shared__ __align__(16) unsigned char dg_smem[];
  double(*sq)[P] = reinterpret_cast<double(*)[P]>(dg_smem);                              // [NQ][P]
  double(*sa)[P] = reinterpret_cast<double(*)[P]>(dg_smem + sizeof(double) * C::NQ * P);  // [9][P]
  double* pf = reinterpret_cast<double*>(dg_smem + sizeof(double) * (C::NQ + kMV + 1) * P);
  __shared__ double sD[3][NP][NP];
  for (int t = threadIdx.x; t < 3 * NP * NP; t += blockDim.x)
    sD[t / (NP * NP)][(t / NP) % NP][t % NP] = tb.Ds[t / (NP * NP)][(t / NP) % NP][t % NP];
  const long long e = blockIdx.x;
  unsigned bad = 0;
  for (int node = threadIdx.x; node < P; node += blockDim.x) {
    double c[kMV];
#pragma unroll
    for (int v = 0; v < kMV; ++v) c[v] = u[(e * kMV + v) * P + node];
    const ECq q = ec_of(mhd_state(c, g.gm1, bad));
    sq[0][node] = q.rho;
    sq[1][node] = q.beta;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sq[2 + k][node] = q.hv[k];
      sq[5 + k][node] = q.hB[k];
    }
    sq[8][node] = q.pm;
    sq[9][node] = q.qv2;
    sq[10][node] = q.qB2;
    sq[11][node] = q.hvB;
#pragma unroll
    for (int v = 0; v <= kMV; ++v) sa[v][node] = 0.0;
  }
  if (bad) atomicOr(err, bad);
  __syncthreads();
  mhd_ec_direction<N, 0>(sq, sa, pf, sD, e, g, tb, fs);
  mhd_ec_direction<N, 1>(sq, sa, pf, sD, e, g, tb, fs);
  mhd_ec_direction<N, 2>(sq, sa, pf, sD, e, g, tb, fs);
  const double dtv = fz.k ? *fz.dt : 0.0;
  double* const uo = fz.u_out ? fz.u_out : u;
  for (int node = threadIdx.x; node < P; node += blockDim.x) {
    double acc[kMV];
#pragma unroll
    for (int v = 0; v < kMV; ++v) acc[v] = sa[v][node];
    if (powell) {
      // Phi = (0, B, v.B, v) from the halved slots: 2 x (hB, hvB, hv)
      const double dn2 = 2.0 * sa[kMV][node];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        acc[1 + k] = fma(sq[5 + k][node], dn2, acc[1 + k]);
        acc[5 + k] = fma(sq[2 + k][node], dn2, acc[5 + k]);
      }
      acc[4] = fma(sq[11][node], dn2, acc[4]);
    }
#pragma unroll
    for (int v = 0; v < kMV; ++v) {
      const long long i = (e * kMV + v) * P + node;
      if (fz.k) {
        double kk = dtv * acc[v];
        if (fz.a != 0.0) kk = fma(fz.a, fz.k[i], kk);
        fz.k[i] = kk;
        uo[i] = u[i] + fz.b * kk;
      } else {
        du[i] = acc[v];
      }
    }
  }
}

__global__ void mhd_speed_kernel(const double* __restrict__ u, Geom g, int P, double s0, double s1,
                                 double s2, unsigned long long* out, unsigned* err,
                                 double* __restrict__ copy_to) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double best = 0.0;
  unsigned bad = 0;
  for (long long e = warp; e < g.nelem; e += nwarps) {
    double lam[3] = {0.0, 0.0, 0.0};
    for (int node = lane; node < P; node += 32) {
      double c[kMV];
#pragma unroll
      for (int v = 0; v < kMV; ++v) c[v] = u[(e * kMV + v) * P + node];
      if (copy_to) {
#pragma unroll
        for (int v = 0; v < kMV; ++v) copy_to[(e * kMV + v) * P + node] = c[v];
      }
      const MState s = mhd_state(c, g.gm1, bad);
      lam[0] = fmax(lam[0], fabs(s.v[0]) + sqrt(fast_speed2<0>(s, g.gamma)));
      lam[1] = fmax(lam[1], fabs(s.v[1]) + sqrt(fast_speed2<1>(s, g.gamma)));
      lam[2] = fmax(lam[2], fabs(s.v[2]) + sqrt(fast_speed2<2>(s, g.gamma)));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int off = 16; off > 0; off >>= 1)
        lam[k] = fmax(lam[k], __shfl_xor_sync(0xffffffffu, lam[k], off));
    double sum = s0 * lam[0];
    sum = sum + s1 * lam[1];
    sum = sum + s2 * lam[2];
    best = fmax(best, sum);
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

// ---- the warped periodic box (the paper's benchmark mesh) ----
// Metric terms Ja[e][r][d][P] = (J a^r)_d and 1/J per node from the curved
// geometry kernel. In direction r a two-point flux is taken along the mean
// of the pair's metric vectors g, f(u; g) = sum_d g_d f_d(u) (every flux
// component is linear in the direction), face fluxes along the metric vector
// of the left element's face node (LLF, HLL in the unit direction scaled by
// |g|, or EC), the Powell divergence as (1/J) times the split-form sums of
// g . (B_i + B_m)/2 and {B} . g, du = (1/J) (...) with the unscaled
// split-form table Ds = -Dt and liftR = -1/w_N, liftL = 1/w_0.

// node quantities of the directional physical flux
struct CMq {
  double m[3], v[3], B[3], Ept, pt, vB;
};

__device__ __forceinline__ CMq cmq_of(const MState& s, const double* c) {
  CMq q;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q.m[k] = c[1 + k];
    q.v[k] = s.v[k];
    q.B[k] = s.B[k];
  }
  q.Ept = s.E + s.pt;
  q.pt = s.pt;
  q.vB = s.vb;
  return q;
}

// f(u; g) = sum_d g_d f_d(u)
__device__ __forceinline__ void mhd_flux_dir(const CMq& q, const double* g, double* f) {
  const double vn = q.v[0] * g[0] + q.v[1] * g[1] + q.v[2] * g[2];
  const double bn = q.B[0] * g[0] + q.B[1] * g[1] + q.B[2] * g[2];
  f[0] = q.m[0] * g[0] + q.m[1] * g[1] + q.m[2] * g[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    f[1 + k] = fma(q.m[k], vn, fma(-q.B[k], bn, q.pt * g[k]));
    f[5 + k] = fma(vn, q.B[k], -bn * q.v[k]);
  }
  f[4] = fma(vn, q.Ept, -bn * q.vB);
}

// EC flux along g (the Cartesian EC flux with its direction replaced by g)
__device__ __forceinline__ void mhd_ec_flux_dir(const ECq& a, const ECq& b, const double* g,
                                                double hgm1inv, double* f) {
  double va[3], Ba[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    va[k] = a.hv[k] + b.hv[k];
    Ba[k] = a.hB[k] + b.hB[k];
  }
  const double vg = va[0] * g[0] + va[1] * g[1] + va[2] * g[2];
  const double bg = Ba[0] * g[0] + Ba[1] * g[1] + Ba[2] * g[2];
  const double rho_ln = ln_mean(a.rho, b.rho);
  const double inv_beta_ln = inv_ln_mean(a.beta, b.beta);
  const double ph = (a.pm + b.pm) / (a.beta + b.beta);
  const double f0 = rho_ln * vg;
  f[0] = f0;
  double e = f0 * fma(hgm1inv, inv_beta_ln, -(a.qv2 + b.qv2));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    f[1 + k] = fma(f0, va[k], fma(-bg, Ba[k], ph * g[k]));
    f[5 + k] = fma(vg, Ba[k], -bg * va[k]);
    e = fma(f[1 + k], va[k], fma(f[5 + k], Ba[k], e));
  }
  e = fma(-vg, a.qB2 + b.qB2, e);
  f[4] = fma(bg, a.hvB + b.hvB, e);
}

// fast magnetosonic speed squared in the unit direction nh
__device__ __forceinline__ double fast_speed2_dir(const MState& s, const double* nh,
                                                  double gamma) {
  const double a2 = gamma * s.p * s.rr;
  const double b2 = s.b2 * s.rr;
  const double bn = s.B[0] * nh[0] + s.B[1] * nh[1] + s.B[2] * nh[2];
  const double bn2 = bn * bn * s.rr;
  const double q = a2 + b2;
  return 0.5 * (q + sqrt(fmax(q * q - 4.0 * a2 * bn2, 0.0)));
}

template <int N, int DIR, int SF>
__device__ __forceinline__ void mhd_curved_surface_body(const double* __restrict__ u,
                                                        const double* __restrict__ Ja,
                                                        double* __restrict__ fs, const Geom& g,
                                                        unsigned& bad) {
  constexpr int NP = N + 1, P = NP * NP * NP, NF = NP * NP;
  const long long total = g.nelem * NF;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / NF;
    const int l = (int)(t % NF);
    const long long er = neighbour(g, e, DIR, +1);
    const int nl = line_node<3, N, DIR>(l, N), nr = line_node<3, N, DIR>(l, 0);
    double cl[kMV], cr[kMV], gv[3];
#pragma unroll
    for (int v = 0; v < kMV; ++v) {
      cl[v] = u[(e * kMV + v) * P + nl];
      cr[v] = u[(er * kMV + v) * P + nr];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) gv[k] = Ja[((e * 3 + DIR) * 3 + k) * P + nl];
    const MState sl = mhd_state(cl, g.gm1, bad), sr = mhd_state(cr, g.gm1, bad);
    const long long base = g.nelem * NF;
    const long long off = e * NF + l;
    double F[kMV];
    if (SF == kMhdEc) {
      mhd_ec_flux_dir(ec_of(sl), ec_of(sr), gv, 0.5 * g.gm1inv, F);
    } else {
      double fl[kMV], fr[kMV];
      mhd_flux_dir(cmq_of(sl, cl), gv, fl);
      mhd_flux_dir(cmq_of(sr, cr), gv, fr);
      const double gn = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
      const double ign = 1.0 / gn;
      const double nh[3] = {gv[0] * ign, gv[1] * ign, gv[2] * ign};
      const double vl = sl.v[0] * nh[0] + sl.v[1] * nh[1] + sl.v[2] * nh[2];
      const double vr = sr.v[0] * nh[0] + sr.v[1] * nh[1] + sr.v[2] * nh[2];
      if (SF == kMhdHll) {
        const double csl = sqrt(fast_speed2_dir(sl, nh, g.gamma));
        const double csr = sqrt(fast_speed2_dir(sr, nh, g.gamma));
        const double sL = fmin(vl - csl, vr - csr), sR = fmax(vl + csl, vr + csr);
        const double inv = 1.0 / (sR - sL);
#pragma unroll
        for (int v = 0; v < kMV; ++v) {
          if (sL >= 0.0) F[v] = fl[v];
          else if (sR <= 0.0) F[v] = fr[v];
          else F[v] = (sR * fl[v] - sL * fr[v] + sL * sR * gn * (cr[v] - cl[v])) * inv;
        }
      } else {
        const double lam = fmax(fabs(vl), fabs(vr)) +
                           sqrt(fmax(fast_speed2_dir(sl, nh, g.gamma),
                                     fast_speed2_dir(sr, nh, g.gamma)));
#pragma unroll
        for (int v = 0; v < kMV; ++v) F[v] = 0.5 * (fl[v] + fr[v]) - 0.5 * lam * gn * (cr[v] - cl[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < kMV; ++v) fs[(long long)(DIR * kMQ + v) * base + off] = F[v];
    fs[(long long)(DIR * kMQ + 8) * base + off] =
        0.5 * ((cl[5] + cr[5]) * gv[0] + (cl[6] + cr[6]) * gv[1] + (cl[7] + cr[7]) * gv[2]);
  }
}

template <int N, int SF>
__global__ void mhd_curved_surface_kernel(const double* __restrict__ u,
                                          const double* __restrict__ Ja, double* __restrict__ fs,
                                          Geom g, unsigned* __restrict__ err) {
  unsigned bad = 0;
  if (blockIdx.y == 0) mhd_curved_surface_body<N, 0, SF>(u, Ja, fs, g, bad);
  else if (blockIdx.y == 1) mhd_curved_surface_body<N, 1, SF>(u, Ja, fs, g, bad);
  else mhd_curved_surface_body<N, 2, SF>(u, Ja, fs, g, bad);
  if (bad) atomicOr(err, bad);
}

// Volume: one element per CTA, the pair-parallel scheme of the EC kernel;
// each thread owns at most one node (THREADS >= P for N <= 7), so the node
// sums stay in registers across the three directions.
template <int N>
struct MCPairs {
  static constexpr int NP = N + 1, P = NP * NP * NP, LINES = NP * NP;
  static constexpr int NPAIRS = N * (N + 1) / 2;
  static constexpr int WORK = LINES * NPAIRS;
  static constexpr int MAXW = WORK > P ? WORK : P;
  static constexpr int THREADS = MAXW < 512 ? ((MAXW + 31) / 32) * 32 : 512;
  static constexpr int NQ = 12;  // ECq slots (EC) or CMq slots (central)
  static constexpr int SMEM = (NQ + 3) * P * (int)sizeof(double) + WORK * kMQ * (int)sizeof(double);
  static_assert(THREADS >= P, "one node per thread");
};

template <int N, int VF>
__device__ __forceinline__ void cq_store(double (*sq)[(N + 1) * (N + 1) * (N + 1)], int n,
                                         const MState& s, const double* c) {
  if (VF == 1) {
    const ECq q = ec_of(s);
    sq[0][n] = q.rho;
    sq[1][n] = q.beta;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sq[2 + k][n] = q.hv[k];
      sq[5 + k][n] = q.hB[k];
    }
    sq[8][n] = q.pm;
    sq[9][n] = q.qv2;
    sq[10][n] = q.qB2;
    sq[11][n] = q.hvB;
  } else {
    const CMq q = cmq_of(s, c);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sq[k][n] = q.m[k];
      sq[3 + k][n] = q.v[k];
      sq[6 + k][n] = q.B[k];
    }
    sq[9][n] = q.Ept;
    sq[10][n] = q.pt;
    sq[11][n] = q.vB;
  }
}

template <int N>
__device__ __forceinline__ CMq cmq_load(const double (*sq)[(N + 1) * (N + 1) * (N + 1)], int n) {
  CMq q;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q.m[k] = sq[k][n];
    q.v[k] = sq[3 + k][n];
    q.B[k] = sq[6 + k][n];
  }
  q.Ept = sq[9][n];
  q.pt = sq[10][n];
  q.vB = sq[11][n];
  return q;
}

template <int N, int VF>
__global__ void __launch_bounds__(MCPairs<N>::THREADS)
    mhd_curved_volume_kernel(double* u, double* __restrict__ du, const double* __restrict__ fs,
                             const double* __restrict__ Ja, const double* __restrict__ invJ,
                             Geom g, CTables tb, int powell, unsigned* __restrict__ err,
                             StageFuse fz) {
  using C = MCPairs<N>;
  constexpr int NP = C::NP, P = C::P, LINES = C::LINES, NPAIRS = C::NPAIRS;
  extern __shared__ __align__(16) unsigned char dg_smem[];
  double(*sq)[P] = reinterpret_cast<double(*)[P]>(dg_smem);                              // [NQ][P]
  double(*sg)[P] = reinterpret_cast<double(*)[P]>(dg_smem + sizeof(double) * C::NQ * P);  // [3][P]
  double* pf = reinterpret_cast<double*>(dg_smem + sizeof(double) * (C::NQ + 3) * P);  // [9][WORK]
  __shared__ double sD[NP][NP];
  for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sD[t / NP][t % NP] = tb.Ds[t / NP][t % NP];
  const long long e = blockIdx.x;
  const int node = threadIdx.x;
  const bool owner = node < P;
  unsigned bad = 0;
  double c[kMV];
  MState s;
  if (owner) {
#pragma unroll
    for (int v = 0; v < kMV; ++v) c[v] = u[(e * kMV + v) * P + node];
    s = mhd_state(c, g.gm1, bad);
    cq_store<N, VF>(sq, node, s, c);
  }
  if (bad) atomicOr(err, bad);
  double acc[kMV], dn = 0.0;
#pragma unroll
  for (int v = 0; v < kMV; ++v) acc[v] = 0.0;
  const long long base = g.nelem * LINES;
  const double hgm1inv = 0.5 * g.gm1inv;
#pragma unroll 1
  for (int r = 0; r < 3; ++r) {
    if (owner) {
#pragma unroll
      for (int k = 0; k < 3; ++k) sg[k][node] = 0.5 * Ja[((e * 3 + r) * 3 + k) * P + node];
    }
    __syncthreads();
    for (int w = threadIdx.x; w < C::WORK; w += blockDim.x) {
      const int l = w / NPAIRS;
      int a, b;
      pair_of<N>(w % NPAIRS, a, b);
      const int na = line_node_rt<3, N>(r, l, a), nb = line_node_rt<3, N>(r, l, b);
      const double gv[3] = {sg[0][na] + sg[0][nb], sg[1][na] + sg[1][nb], sg[2][na] + sg[2][nb]};
      double f[kMV], bb;
      if (VF == 1) {
        const ECq qa = ec_load<N>(sq, na), qb = ec_load<N>(sq, nb);
        mhd_ec_flux_dir(qa, qb, gv, hgm1inv, f);
        bb = (qa.hB[0] + qb.hB[0]) * gv[0] + (qa.hB[1] + qb.hB[1]) * gv[1] +
             (qa.hB[2] + qb.hB[2]) * gv[2];
      } else {
        const CMq qa = cmq_load<N>(sq, na), qb = cmq_load<N>(sq, nb);
        double fa[kMV], fb[kMV];
        mhd_flux_dir(qa, gv, fa);
        mhd_flux_dir(qb, gv, fb);
#pragma unroll
        for (int v = 0; v < kMV; ++v) f[v] = 0.5 * (fa[v] + fb[v]);
        bb = 0.5 * ((qa.B[0] + qb.B[0]) * gv[0] + (qa.B[1] + qb.B[1]) * gv[1] +
                    (qa.B[2] + qb.B[2]) * gv[2]);
      }
#pragma unroll
      for (int v = 0; v < kMV; ++v) pf[v * C::WORK + w] = f[v];
      pf[kMV * C::WORK + w] = bb;
    }
    __syncthreads();
    if (owner) {
      int l, i;
      line_of<N>(r, node, l, i);
      for (int j = 0; j < NP; ++j) {
        if (j == i) continue;
        const int p = j < i ? pair_index<N>(j, i) : pair_index<N>(i, j);
        const double dij = sD[i][j];
#pragma unroll
        for (int v = 0; v < kMV; ++v) acc[v] = fma(dij, pf[v * C::WORK + l * NPAIRS + p], acc[v]);
        dn = fma(dij, pf[kMV * C::WORK + l * NPAIRS + p], dn);
      }
      if (i == N || i == 0) {
        const long long ef = i == N ? e : neighbour(g, e, r, -1);
        const double lift = i == N ? tb.liftR : tb.liftL;
        const double* src = fs + (long long)r * kMQ * base + ef * LINES + l;
#pragma unroll
        for (int v = 0; v < kMV; ++v) acc[v] = fma(lift, src[v * base], acc[v]);
        dn = fma(lift, src[8 * base], dn);
      }
    }
    __syncthreads();
  }
  if (!owner) return;
  if (powell) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc[1 + k] = fma(s.B[k], dn, acc[1 + k]);
      acc[5 + k] = fma(s.v[k], dn, acc[5 + k]);
    }
    acc[4] = fma(s.vb, dn, acc[4]);
  }
  const double ij = invJ[e * P + node];
  const double dtv = fz.k ? *fz.dt : 0.0;
  double* const uo = fz.u_out ? fz.u_out : u;
#pragma unroll
  for (int v = 0; v < kMV; ++v) {
    const long long i = (e * kMV + v) * P + node;
    const double val = ij * acc[v];
    if (fz.k) {
      double kk = dtv * val;
      if (fz.a != 0.0) kk = fma(fz.a, fz.k[i], kk);
      fz.k[i] = kk;
      uo[i] = c[v] + fz.b * kk;
    } else {
      du[i] = val;
    }
  }
}

// per element sum_r max_nodes (|v . J a^r| + c_f(a^r) |J a^r|) / J, max over
// elements (ordered bits)
__global__ void mhd_curved_speed_kernel(const double* __restrict__ u,
                                        const double* __restrict__ Ja,
                                        const double* __restrict__ invJ, Geom g, int P,
                                        unsigned long long* out, unsigned* err,
                                        double* __restrict__ copy_to) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double best = 0.0;
  unsigned bad = 0;
  for (long long e = warp; e < g.nelem; e += nwarps) {
    double lam[3] = {0.0, 0.0, 0.0};
    for (int node = lane; node < P; node += 32) {
      double c[kMV];
#pragma unroll
      for (int v = 0; v < kMV; ++v) c[v] = u[(e * kMV + v) * P + node];
      if (copy_to) {
#pragma unroll
        for (int v = 0; v < kMV; ++v) copy_to[(e * kMV + v) * P + node] = c[v];
      }
      const MState s = mhd_state(c, g.gm1, bad);
      const double ij = invJ[e * P + node];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        double gv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) gv[k] = Ja[((e * 3 + r) * 3 + k) * P + node];
        const double gn = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
        const double nh[3] = {gv[0] / gn, gv[1] / gn, gv[2] / gn};
        const double vg = s.v[0] * gv[0] + s.v[1] * gv[1] + s.v[2] * gv[2];
        lam[r] = fmax(lam[r], (fabs(vg) + sqrt(fast_speed2_dir(s, nh, g.gamma)) * gn) * ij);
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int off = 16; off > 0; off >>= 1)
        lam[k] = fmax(lam[k], __shfl_xor_sync(0xffffffffu, lam[k], off));
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

template <int N>
cudaError_t mhd_curved_rhs_n(const double* u, double* du, double* fs, const double* Ja,
                             const double* invJ, const Geom& g, const CTables& tb, int vf,
                             int powell, int sf, unsigned* err, cudaStream_t st, int parts,
                             const StageFuse& fz) {
  constexpr int NF = (N + 1) * (N + 1);
  if (parts & 1) {
    const long long total = g.nelem * NF;
    const int threads = (total < 152LL * 4 * 256) ? 64 : 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    const dim3 grid((unsigned)blocks, 3);
    if (sf == kMhdHll)
      mhd_curved_surface_kernel<N, kMhdHll><<<grid, threads, 0, st>>>(u, Ja, fs, g, err);
    else if (sf == kMhdEc)
      mhd_curved_surface_kernel<N, kMhdEc><<<grid, threads, 0, st>>>(u, Ja, fs, g, err);
    else
      mhd_curved_surface_kernel<N, kMhdLlf><<<grid, threads, 0, st>>>(u, Ja, fs, g, err);
  }
  if (!(parts & 2)) return cudaGetLastError();
  using C = MCPairs<N>;
  cudaError_t e;
  if (vf == 1) {
    auto kern = mhd_curved_volume_kernel<N, 1>;
    if (C::SMEM > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM)) !=
            cudaSuccess)
      return e;
    kern<<<(unsigned)g.nelem, C::THREADS, C::SMEM, st>>>(const_cast<double*>(u), du, fs, Ja,
                                                          invJ, g, tb, powell, err, fz);
  } else {
    auto kern = mhd_curved_volume_kernel<N, 0>;
    if (C::SMEM > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM)) !=
            cudaSuccess)
      return e;
    kern<<<(unsigned)g.nelem, C::THREADS, C::SMEM, st>>>(const_cast<double*>(u), du, fs, Ja,
                                                          invJ, g, tb, powell, err, fz);
  }
  return cudaGetLastError();
}

// elements per CTA: about kMhdThreads threads
template <int N>
struct MLaunch {
  static constexpr int P = (N + 1) * (N + 1) * (N + 1);
  static constexpr int EPB = (kMhdThreads / P) > 0 ? (kMhdThreads / P) : 1;
};

template <int N, int EPB>
cudaError_t mhd_volume_epb(const double* u, double* du, const double* fs, const Geom& g,
                           const Tables<double>& tb, int powell, unsigned* err, cudaStream_t st,
                           const StageFuse& fz) {
  constexpr int P = MLaunch<N>::P;
  constexpr int SMEM = EPB * kMV * P * (int)sizeof(double);
  auto kern = mhd_volume_kernel<N, EPB>;
  if (SMEM > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
  }
  const long long grid = (g.nelem + EPB - 1) / EPB;
  kern<<<(unsigned)grid, EPB * P, SMEM, st>>>(const_cast<double*>(u), du, fs, g, tb, powell, err,
                                               fz);
  return cudaGetLastError();
}

template <int N>
cudaError_t mhd_volume_ec(const double* u, double* du, const double* fs, const Geom& g,
                          const Tables<double>& tdt, int powell, unsigned* err, cudaStream_t st,
                          const StageFuse& fz) {
  using C = MPairs<N>;
  auto kern = mhd_volume_ec_kernel<N>;
  if (C::SMEM > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
  }
  kern<<<(unsigned)g.nelem, C::THREADS, C::SMEM, st>>>(const_cast<double*>(u), du, fs, g, tdt,
                                                        powell, err, fz);
  return cudaGetLastError();
}

template <int N>
cudaError_t mhd_rhs_n(const double* u, double* du, double* fs, const Geom& g,
                      const Tables<double>& tb, const Tables<double>& tdt, int vf, int powell,
                      int sf, unsigned* err, cudaStream_t st, int parts, const StageFuse& fz) {
  constexpr int NF = (N + 1) * (N + 1);
  if (parts & 1) {
    const long long total = g.nelem * NF;
    const int threads = (total < 152LL * 4 * 256) ? 64 : 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (sf == kMhdHll)
      mhd_surface_kernel<N, kMhdHll><<<dim3((unsigned)blocks, 3), threads, 0, st>>>(u, fs, g, err);
    else if (sf == kMhdEc)
      mhd_surface_kernel<N, kMhdEc><<<dim3((unsigned)blocks, 3), threads, 0, st>>>(u, fs, g, err);
    else
      mhd_surface_kernel<N, kMhdLlf><<<dim3((unsigned)blocks, 3), threads, 0, st>>>(u, fs, g, err);
  }
  if (!(parts & 2)) return cudaGetLastError();
  if (vf == 1) return mhd_volume_ec<N>(u, du, fs, g, tdt, powell, err, st, fz);
  constexpr int EPB = MLaunch<N>::EPB;
  if (EPB > 1 && g.nelem < 2LL * 152 * EPB)
    return mhd_volume_epb<N, 1>(u, du, fs, g, tb, powell, err, st, fz);
  return mhd_volume_epb<N, EPB>(u, du, fs, g, tb, powell, err, st, fz);
}

}  // namespace

cudaError_t mhd_rhs_launch(int N, const double* u, double* du, double* fs, const Geom& g,
                           const Tables<double>& tb, const Tables<double>& tdt, int vf,
                           int powell, int sf, unsigned* err, cudaStream_t st, int parts,
                           const StageFuse& fz) {
  switch (N) {
    case 1: return mhd_rhs_n<1>(u, du, fs, g, tb, tdt, vf, powell, sf, err, st, parts, fz);
    case 2: return mhd_rhs_n<2>(u, du, fs, g, tb, tdt, vf, powell, sf, err, st, parts, fz);
    case 3: return mhd_rhs_n<3>(u, du, fs, g, tb, tdt, vf, powell, sf, err, st, parts, fz);
    case 4: return mhd_rhs_n<4>(u, du, fs, g, tb, tdt, vf, powell, sf, err, st, parts, fz);
    case 5: return mhd_rhs_n<5>(u, du, fs, g, tb, tdt, vf, powell, sf, err, st, parts, fz);
    case 6: return mhd_rhs_n<6>(u, du, fs, g, tb, tdt, vf, powell, sf, err, st, parts, fz);
    case 7: return mhd_rhs_n<7>(u, du, fs, g, tb, tdt, vf, powell, sf, err, st, parts, fz);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t mhd_curved_rhs_launch(int N, const double* u, double* du, double* fs, const double* Ja,
                                  const double* invJ, const Geom& g, const CTables& tb, int vf,
                                  int powell, int sf, unsigned* err, cudaStream_t st, int parts,
                                  const StageFuse& fz) {
  switch (N) {
#define DG_MC(n) \
  case n:        \
    return mhd_curved_rhs_n<n>(u, du, fs, Ja, invJ, g, tb, vf, powell, sf, err, st, parts, fz);
    DG_MC(1)
    DG_MC(2)
    DG_MC(3)
    DG_MC(4)
    DG_MC(5)
    DG_MC(6)
    DG_MC(7)
#undef DG_MC
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t mhd_curved_speed_launch(const double* u, const double* Ja, const double* invJ,
                                    const Geom& g, int P, unsigned long long* out, unsigned* err,
                                    double* copy_to, int grid, int threads, cudaStream_t st) {
  mhd_curved_speed_kernel<<<grid, threads, 0, st>>>(u, Ja, invJ, g, P, out, err, copy_to);
  return cudaGetLastError();
}

cudaError_t mhd_speed_launch(const double* u, const Geom& g, int P, const double* s,
                             unsigned long long* out, unsigned* err, double* copy_to, int grid,
                             int threads, cudaStream_t st) {
  mhd_speed_kernel<<<grid, threads, 0, st>>>(u, g, P, s[0], s[1], s[2], out, err, copy_to);
  return cudaGetLastError();
}

}  // namespace dg
