// Batched ensemble of independent 3D periodic Euler simulations with uneven
// mesh sizes and polynomial degrees (N in {3, 4, 5}), advanced together:
// one persistent kernel launch per Runge-Kutta stage over a work list of
// (simulation, element batch) items, a graph-capturable step (the per-
// simulation time steps stay on the device) and an autotuner that picks the
// CTA size (hence the elements per CTA for every degree).
//
// Each work item evaluates, for its elements, the surface fluxes on all
// element faces (reading the neighbours' traces; the two elements of a face
// evaluate the same F* from the same inputs), the flux-differencing volume
// term, the lifting, and the stage update k <- A k + dt du, u_out <- u_in + B k.
// The stage reads u_in and writes u_out (two buffers), so no element waits
// for another inside a launch. Arithmetic as in dg_rhs (same formulas,
// tables unscaled and multiplied by -2/h per node at the end).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dgsem.h"
#include "dg_rhs_kernels.cuh"

namespace dg {
int set_last_error(int code, const char* msg);
}

namespace {

using namespace dg;

constexpr int kEnsMinN = 3, kEnsMaxN = 5;

struct SimDesc {
  int N, n, nelem;
  long long off;  // offset of the simulation's first value
  double s;       // -2/h
  double lam_scale;  // 2/h (for the wave-speed sum)
};

struct WorkItem {
  int sim, e0, count;
};

// unscaled split-form matrices and inverse boundary weights per degree
struct EnsTables {
  double Dt[kEnsMaxN - kEnsMinN + 1][8][8];
  double iw0[kEnsMaxN - kEnsMinN + 1];  // 1 / w_0 (= 1 / w_N)
};

struct EnsArgs {
  const SimDesc* sims;
  const WorkItem* items;
  int nitems;
  const double* uin;
  double* uout;
  double* k;
  const double* dt;  // per simulation
  double A, B;
  double gamma, gm1, gm1inv;
  int sf;
  unsigned* err;
};

int fail(int code, const char* msg) { return dg::set_last_error(code, msg); }

template <int N>
struct EShape {
  static constexpr int NP = N + 1, P = NP * NP * NP, LINES = NP * NP, NC = 9;
};

// conserved trace of node `node` of element e -> Trace (normal-first) with ps
// relative to the pressure reference Pown (FP32) or p itself (FP64)
template <typename R>
__device__ __forceinline__ void load_trace(const double* __restrict__ u, long long base, int P,
                                           int node, int dir, double gm1, float Pown, double* c,
                                           Trace<R, 3>& T) {
#pragma unroll
  for (int v = 0; v < 5; ++v) c[v] = u[base + (long long)v * P + node];
  const int t1 = (dir + 1) % 3, t2 = (dir + 2) % 3;
  if (sizeof(R) == 4) {
    // the node's own element reference: E at its first node
    const double Er = u[base + 4LL * P];
    const double pe = gm1 * Er;
    const float Pe = (float)pe, ce = (float)(pe - (double)Pe);
    float rho, v[3], pp, p;
    prim_f32<3>(c, (float)gm1, Pe, ce, Er, rho, v, pp, p);
    T.rho = R(rho);
    T.rr = R(rcp(rho));
    T.p = R(p);
    T.ps = R(pp + (Pe - Pown));
    T.vn = R(v[dir]);
    T.vt[0] = R(v[t1]);
    T.vt[1] = R(v[t2]);
  } else {
    double rr;
    const Prim<double, 3> q = prim_rcp<3>(c, gm1, rr);
    T.rho = R(q.rho);
    T.rr = R(rr);
    T.p = R(q.p);
    T.ps = T.p;
    T.vn = R(q.v[dir]);
    T.vt[0] = R(q.v[t1]);
    T.vt[1] = R(q.v[t2]);
  }
  T.mn = R(c[1 + dir]);
  T.mt[0] = R(c[1 + t1]);
  T.mt[1] = R(c[1 + t2]);
  T.E = R(c[4]);
}

template <typename R, int N>
__device__ void ens_process(const EnsArgs& a, const SimDesc& sd, int sim, int e0, int count,
                            const EnsTables& et, unsigned char* smem) {
  using S = EShape<N>;
  constexpr int NP = S::NP, P = S::P, LINES = S::LINES, NV = 5, NC = S::NC;
  constexpr bool F32 = sizeof(R) == 4;
  R(*sp)[NC][P] = reinterpret_cast<R(*)[NC][P]>(smem);
  R(*sa)[6][P] = reinterpret_cast<R(*)[6][P]>(smem + sizeof(R) * count * NC * P);
  __shared__ int s_nb[32][3][2];
  __shared__ float s_pe[32], s_ce[32];
  __shared__ double s_er[32];
  const int n = sd.n;
  const R gm1inv = R(a.gm1inv);
  const double* u = a.uin + sd.off;
  if ((int)threadIdx.x < count) {
    const int el = threadIdx.x, e = e0 + el;
    const int x = e % n, r = e / n, y = r % n, z = r / n;
    s_nb[el][0][0] = ((x + n - 1) % n) + n * (y + n * z);
    s_nb[el][0][1] = ((x + 1) % n) + n * (y + n * z);
    s_nb[el][1][0] = x + n * (((y + n - 1) % n) + n * z);
    s_nb[el][1][1] = x + n * (((y + 1) % n) + n * z);
    s_nb[el][2][0] = x + n * (y + n * ((z + n - 1) % n));
    s_nb[el][2][1] = x + n * (y + n * ((z + 1) % n));
    const double Er = u[((long long)e * NV + 4) * P];
    const double pe = a.gm1 * Er;
    s_pe[el] = (float)pe;
    s_ce[el] = (float)(pe - (double)(float)pe);
    s_er[el] = Er;
  }
  __syncthreads();
  unsigned bad = 0;
  for (int t = threadIdx.x; t < count * P; t += blockDim.x) {
    const int el = t / P, node = t % P, e = e0 + el;
    double c[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = u[((long long)e * NV + v) * P + node];
    R rho, p, hp, vv[3];
    if (F32) {
      float vf[3], pp, pf, rf;
      prim_f32<3>(c, (float)a.gm1, s_pe[el], s_ce[el], s_er[el], rf, vf, pp, pf);
      rho = R(rf);
      p = R(pf);
      hp = R(0.5f * pp);
#pragma unroll
      for (int k = 0; k < 3; ++k) vv[k] = R(vf[k]);
      if (!(rf > 0.0f)) bad |= kErrRho;
      if (!(pf > 0.0f)) bad |= kErrP;
      if (!isfinite(rf) || !isfinite(pf)) bad |= kErrNaN;
    } else {
      double rr;
      const Prim<double, 3> q = prim_rcp<3>(c, a.gm1, rr);
      bad |= prim_check(q);
      rho = R(q.rho);
      p = R(q.p);
      hp = R(0.5) * p;
#pragma unroll
      for (int k = 0; k < 3; ++k) vv[k] = R(q.v[k]);
    }
    node_slots<kVRanocha, R>(rho, p, R(a.gm1), sp[el][0][node], sp[el][1][node]);
    sp[el][2][node] = hp;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sp[el][3 + k][node] = vv[k];
      sp[el][6 + k][node] = R(0.5) * vv[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) sa[el][k][node] = R(0);
  }
  if (bad) atomicOr(a.err, bad);
  __syncthreads();
  const int el = threadIdx.x / LINES, l = threadIdx.x % LINES;
  const bool active = el < count;
  const R iw = R(et.iw0[N - kEnsMinN]);
#pragma unroll 1
  for (int dir = 0; dir < 3; ++dir) {
    if (active) {
      const int e = e0 + el;
      const int t1 = (dir + 1) % 3, t2 = (dir + 2) % 3;
      int node[NP];
      LinePrim<R, 3> q[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        node[i] = line_node_rt<3, N>(dir, l, i);
        const int nd = node[i];
        q[i].s0 = sp[el][0][nd];
        q[i].s1 = sp[el][1][nd];
        q[i].hp = sp[el][2][nd];
        q[i].vn = sp[el][3 + dir][nd];
        q[i].hvn = sp[el][6 + dir][nd];
        q[i].vt[0] = sp[el][3 + t1][nd];
        q[i].hvt[0] = sp[el][6 + t1][nd];
        q[i].vt[1] = sp[el][3 + t2][nd];
        q[i].hvt[1] = sp[el][6 + t2][nd];
      }
      constexpr int NA = F32 ? 6 : 5;
      R acc[NP][NA];
#pragma unroll
      for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int v = 0; v < NA; ++v) acc[i][v] = R(0);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
#pragma unroll
        for (int j = i + 1; j < NP; ++j) {
          R f[NV], an;
          ranocha_nf<R, 3>(q[i], q[j], f, an);
          const R dij = R(et.Dt[N - kEnsMinN][i][j]), dji = R(et.Dt[N - kEnsMinN][j][i]);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            acc[i][v] = fma(dij, f[v], acc[i][v]);
            acc[j][v] = fma(dji, f[v], acc[j][v]);
          }
          if (F32) {
            acc[i][NA - 1] = fma(dij, an, acc[i][NA - 1]);
            acc[j][NA - 1] = fma(dji, an, acc[j][NA - 1]);
          }
        }
      }
      // the two faces at the ends of this line: left (node 0) and right (node N)
      {
        const long long base_e = sd.off + (long long)e * NV * P;
        const int eL = s_nb[el][dir][0], eR = s_nb[el][dir][1];
        double cn[NV], co[NV];
        Trace<R, 3> TL, TO, TR;
        R f[NV];
        const float Pown = F32 ? s_pe[el] : 0.0f;
        load_trace<R>(a.uin, sd.off + (long long)eL * NV * P, P, line_node_rt<3, N>(dir, l, N), dir,
                      a.gm1, Pown, cn, TL);
        load_trace<R>(a.uin, base_e, P, node[0], dir, a.gm1, Pown, co, TO);
        surface_nf<R, 3>(a.sf, TL, TO, R(co[4] - cn[4]), R(a.gamma), gm1inv, f);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[0][v] = fma(-iw, f[v], acc[0][v]);
        load_trace<R>(a.uin, base_e, P, node[N], dir, a.gm1, Pown, co, TO);
        load_trace<R>(a.uin, sd.off + (long long)eR * NV * P, P, line_node_rt<3, N>(dir, l, 0), dir,
                      a.gm1, Pown, cn, TR);
        surface_nf<R, 3>(a.sf, TO, TR, R(cn[4] - co[4]), R(a.gamma), gm1inv, f);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[N][v] = fma(iw, f[v], acc[N][v]);
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const int nd = node[i];
        sa[el][0][nd] += acc[i][0];
        sa[el][1 + dir][nd] += acc[i][1];
        sa[el][1 + t1][nd] += acc[i][2];
        sa[el][1 + t2][nd] += acc[i][3];
        sa[el][4][nd] += acc[i][4];
        if (F32) sa[el][5][nd] += acc[i][NA - 1];
      }
    }
    __syncthreads();
  }
  // epilogue: du = -(2/h) (volume + surface); stage update
  const double dt = a.dt[sim];
  for (int t = threadIdx.x; t < count * P; t += blockDim.x) {
    const int ell = t / P, node = t % P, e = e0 + ell;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      R val = sa[ell][v][node];
      if (F32 && v == 4) val = fma(R(s_pe[ell]), sa[ell][5][node], val);
      const double du = sd.s * (double)val;
      const long long i = sd.off + ((long long)e * NV + v) * P + node;
      double kk = dt * du;
      if (a.A != 0.0) kk = fma(a.A, a.k[i], kk);  // the first stage reads no k
      a.k[i] = kk;
      a.uout[i] = a.uin[i] + a.B * kk;
    }
  }
}


// one launch per stage: blocks walk the work list (largest degrees first)
template <typename R>
__global__ void __launch_bounds__(256) ensemble_stage_kernel(EnsArgs a, EnsTables et) {
  extern __shared__ __align__(16) unsigned char dg_smem[];
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const WorkItem w = a.items[it];
    const SimDesc sd = a.sims[w.sim];
    if (sd.N == 3) ens_process<R, 3>(a, sd, w.sim, w.e0, w.count, et, dg_smem);
    else if (sd.N == 4) ens_process<R, 4>(a, sd, w.sim, w.e0, w.count, et, dg_smem);
    else ens_process<R, 5>(a, sd, w.sim, w.e0, w.count, et, dg_smem);
    __syncthreads();
  }
}

// per-simulation max over elements of (2/h) sum_k max_nodes(|v_k| + c),
// stored as ordered bits; then dt_s = cfl 2 / ((N_s + 1) max_s)
__global__ void ensemble_speed_kernel(const SimDesc* __restrict__ sims,
                                      const WorkItem* __restrict__ items, int nitems,
                                      const double* __restrict__ u, double gamma, double gm1,
                                      unsigned long long* __restrict__ smax,
                                      unsigned* __restrict__ err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned bad = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const SimDesc sd = sims[w.sim];
    const int P = (sd.N + 1) * (sd.N + 1) * (sd.N + 1);
    for (int el = warp; el < w.count; el += nw) {
      const long long base = sd.off + (long long)(w.e0 + el) * 5 * P;
      double lam[3] = {0.0, 0.0, 0.0};
      for (int node = lane; node < P; node += 32) {
        double c[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) c[v] = u[base + (long long)v * P + node];
        double rr;
        const Prim<double, 3> q = prim_rcp<3>(c, gm1, rr);
        bad |= prim_check(q);
        const double cs = sqrt(gamma * q.p * rr);
#pragma unroll
        for (int k = 0; k < 3; ++k) lam[k] = fmax(lam[k], fabs(q.v[k]) + cs);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
        for (int off = 16; off > 0; off >>= 1)
          lam[k] = fmax(lam[k], __shfl_xor_sync(0xffffffffu, lam[k], off));
      if (lane == 0) {
        double s = sd.lam_scale * lam[0];
        s = s + sd.lam_scale * lam[1];
        s = s + sd.lam_scale * lam[2];
        atomicMax(&smax[w.sim], (unsigned long long)__double_as_longlong(s));
      }
    }
  }
  if (bad) atomicOr(err, bad);
}

__global__ void ensemble_dt_kernel(const SimDesc* __restrict__ sims, int nsims, double cfl,
                                   unsigned long long* __restrict__ smax,
                                   double* __restrict__ dt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsims) return;
  const double m = __longlong_as_double((long long)smax[s]);
  dt[s] = cfl * 2.0 / ((sims[s].N + 1) * m);
  smax[s] = 0ull;
}

// Carpenter-Kennedy (1994) five-stage fourth-order 2N-storage coefficients
const double kA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                      1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                      2277821191437.0 / 14882151754819.0};

// long double LGL basis for the ensemble's tables (the same construction as
// the single-mesh path: Newton on P_{N+1} - P_{N-1}, closed-form D)
long double leg(int n, long double x) {
  if (n == 0) return 1.0L;
  long double a = 1.0L, b = x;
  for (int k = 1; k < n; ++k) {
    long double c = ((2.0L * k + 1.0L) * x * b - k * a) / (k + 1.0L);
    a = b;
    b = c;
  }
  return b;
}

void ens_basis(int N, double Dt[8][8], double* iw0) {
  const long double pi = 3.14159265358979323846264338327950288L;
  long double x[8], w[8];
  for (int j = 0; j <= N; ++j) {
    long double t = -cosl(pi * j / N);
    if (j > 0 && j < N)
      for (int it = 0; it < 200; ++it) {
        long double step = (leg(N + 1, t) - leg(N - 1, t)) / ((2.0L * N + 1.0L) * leg(N, t));
        t -= step;
        if (fabsl(step) <= 1e-32L) break;
      }
    if (j == 0) t = -1.0L;
    if (j == N) t = 1.0L;
    x[j] = t;
    const long double pn = leg(N, t);
    w[j] = 2.0L / ((long double)N * (N + 1) * pn * pn);
  }
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) {
      long double dij;
      if (i != j) dij = leg(N, x[i]) / (leg(N, x[j]) * (x[i] - x[j]));
      else if (i == 0) dij = -(long double)N * (N + 1) / 4.0L;
      else if (i == N) dij = (long double)N * (N + 1) / 4.0L;
      else dij = 0.0L;
      const long double b = (i == j && i == 0) ? -1.0L : (i == j && i == N) ? 1.0L : 0.0L;
      Dt[i][j] = (double)(2.0L * dij - b / w[i]);
    }
  *iw0 = (double)(1.0L / w[0]);
}

}  // namespace

struct dg_ensemble {
  int nsims;
  dg_options opt;
  cudaStream_t stream;
  std::vector<SimDesc> sims;
  long long nvalues, nnodes;
  int block;  // threads per CTA (tunable)
  int grid;   // persistent blocks
  int nitems;
  SimDesc* d_sims;
  WorkItem* d_items;
  double* k;
  double* dt;
  unsigned long long* smax;
  unsigned* err;
  EnsTables tables;
  cudaGraphExec_t graph;
  const double* graph_u;
  const double* graph_tmp;
  double graph_cfl;
};

namespace {

// elements per work item for degree N with `block` threads per CTA
int items_epb(int N, int block) {
  const int lines = (N + 1) * (N + 1);
  int e = block / lines;
  if (e > 32) e = 32;
  return e < 1 ? 0 : e;
}

int smem_for(int precision, int block) {
  const int rs = precision == DG_FP64 ? 8 : 4;
  int m = 0;
  for (int N = kEnsMinN; N <= kEnsMaxN; ++N) {
    const int P = (N + 1) * (N + 1) * (N + 1);
    const int b = items_epb(N, block) * (9 + 6) * P * rs;  // node slots + accumulators
    if (b > m) m = b;
  }
  return m;
}

int build_items(dg_ensemble* E) {
  std::vector<WorkItem> items;
  for (int N = kEnsMaxN; N >= kEnsMinN; --N) {
    const int epb = items_epb(N, E->block);
    if (epb < 1) return fail(DG_ERR_ARG, "dg_ensemble: CTA too small for the degree");
    for (int s = 0; s < E->nsims; ++s) {
      if (E->sims[s].N != N) continue;
      for (int e0 = 0; e0 < E->sims[s].nelem; e0 += epb)
        items.push_back(WorkItem{s, e0, std::min(epb, E->sims[s].nelem - e0)});
    }
  }
  cudaFree(E->d_items);
  E->d_items = nullptr;
  if (cudaMalloc(&E->d_items, items.size() * sizeof(WorkItem)) != cudaSuccess)
    return fail(DG_ERR_OOM, "dg_ensemble: cudaMalloc of the work list failed");
  if (cudaMemcpy(E->d_items, items.data(), items.size() * sizeof(WorkItem),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble: copying the work list failed");
  E->nitems = (int)items.size();
  return DG_OK;
}

int launch_stage(dg_ensemble* E, const double* uin, double* uout, int s) {
  EnsArgs a;
  a.sims = E->d_sims;
  a.items = E->d_items;
  a.nitems = E->nitems;
  a.uin = uin;
  a.uout = uout;
  a.k = E->k;
  a.dt = E->dt;
  a.A = kA[s];
  a.B = kB[s];
  a.gamma = E->opt.gamma;
  a.gm1 = E->opt.gamma - 1.0;
  a.gm1inv = 1.0 / (E->opt.gamma - 1.0);
  a.sf = E->opt.surface_flux;
  a.err = E->err;
  const int sm = smem_for(E->opt.precision, E->block);
  cudaError_t e;
  if (E->opt.precision == DG_FP64) {
    if ((e = allow_smem(ensemble_stage_kernel<double>, sm)) != cudaSuccess)
      return fail(DG_ERR_CUDA, "dg_ensemble: shared-memory attribute");
    ensemble_stage_kernel<double><<<E->grid, E->block, sm, E->stream>>>(a, E->tables);
  } else {
    if ((e = allow_smem(ensemble_stage_kernel<float>, sm)) != cudaSuccess)
      return fail(DG_ERR_CUDA, "dg_ensemble: shared-memory attribute");
    ensemble_stage_kernel<float><<<E->grid, E->block, sm, E->stream>>>(a, E->tables);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(DG_ERR_CUDA, cudaGetErrorString(e));
  return DG_OK;
}

int launch_dt(dg_ensemble* E, const double* u, double cfl) {
  ensemble_speed_kernel<<<E->grid, 256, 0, E->stream>>>(E->d_sims, E->d_items, E->nitems, u,
                                                         E->opt.gamma, E->opt.gamma - 1.0,
                                                         E->smax, E->err);
  ensemble_dt_kernel<<<(E->nsims + 127) / 128, 128, 0, E->stream>>>(E->d_sims, E->nsims, cfl,
                                                                    E->smax, E->dt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, cudaGetErrorString(e));
  return DG_OK;
}

// one step: (dt from u when cfl > 0), five stages alternating u -> tmp -> u
// ..., ending in tmp, then tmp copied back to u
int enqueue_step(dg_ensemble* E, double* u, double* tmp, double cfl) {
  int rc = (cfl > 0.0) ? launch_dt(E, u, cfl) : DG_OK;
  if (rc) return rc;
  const double* in = u;
  double* out = tmp;
  for (int s = 0; s < 5; ++s) {
    rc = launch_stage(E, in, out, s);
    if (rc) return rc;
    double* nxt = (out == tmp) ? u : tmp;
    in = out;
    out = nxt;
  }
  if (cudaMemcpyAsync(u, tmp, E->nvalues * sizeof(double), cudaMemcpyDeviceToDevice,
                      E->stream) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble: copy of the step result failed");
  return DG_OK;
}

}  // namespace

extern "C" {

int dg_ensemble_destroy(dg_ensemble* E) {
  if (!E) return DG_OK;
  cudaStreamSynchronize(E->stream);
  if (E->graph) cudaGraphExecDestroy(E->graph);
  cudaFree(E->d_sims);
  cudaFree(E->d_items);
  cudaFree(E->k);
  cudaFree(E->dt);
  cudaFree(E->smax);
  cudaFree(E->err);
  delete E;
  return DG_OK;
}

int dg_ensemble_create(int n_sims, const int* N, const int* elements_per_dim,
                       const dg_options* opt, void* cuda_stream, dg_ensemble** out) {
  if (out) *out = nullptr;
  if (!out || !N || !elements_per_dim || n_sims < 1)
    return fail(DG_ERR_ARG, "dg_ensemble_create: bad arguments");
  dg_options o = {1.4, DG_VFLUX_RANOCHA, DG_SFLUX_LLF, DG_FP64};
  if (opt) o = *opt;
  if (!(o.gamma > 1.0) || o.volume_flux != DG_VFLUX_RANOCHA || o.surface_flux < 0 ||
      o.surface_flux > 3 || (o.precision != DG_FP64 && o.precision != DG_FP32))
    return fail(DG_ERR_ARG, "dg_ensemble_create: invalid options (Ranocha volume flux only)");
  for (int s = 0; s < n_sims; ++s)
    if (N[s] < kEnsMinN || N[s] > kEnsMaxN || elements_per_dim[s] < 1 ||
        elements_per_dim[s] > 1024)
      return fail(DG_ERR_ARG, "dg_ensemble_create: N must be in {3,4,5} and 1 <= n <= 1024");
  dg_ensemble* E = new dg_ensemble();
  E->nsims = n_sims;
  E->opt = o;
  E->stream = (cudaStream_t)cuda_stream;
  E->block = 128;
  E->d_sims = nullptr;
  E->d_items = nullptr;
  E->k = nullptr;
  E->dt = nullptr;
  E->smax = nullptr;
  E->err = nullptr;
  E->graph = nullptr;
  E->graph_u = E->graph_tmp = nullptr;
  E->graph_cfl = 0.0;
  long long off = 0, nodes = 0;
  for (int s = 0; s < n_sims; ++s) {
    SimDesc sd;
    sd.N = N[s];
    sd.n = elements_per_dim[s];
    sd.nelem = sd.n * sd.n * sd.n;
    sd.off = off;
    const double h = 2.0 / sd.n;  // every member lives on [-1, 1]^3
    sd.s = -2.0 / h;
    sd.lam_scale = 2.0 / h;
    const long long P = (long long)(sd.N + 1) * (sd.N + 1) * (sd.N + 1);
    off += 5LL * sd.nelem * P;
    nodes += sd.nelem * P;
    E->sims.push_back(sd);
  }
  E->nvalues = off;
  E->nnodes = nodes;
  memset(&E->tables, 0, sizeof(E->tables));
  for (int n = kEnsMinN; n <= kEnsMaxN; ++n)
    ens_basis(n, E->tables.Dt[n - kEnsMinN], &E->tables.iw0[n - kEnsMinN]);
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  E->grid = nsm * 4;
  if (cudaMalloc(&E->d_sims, n_sims * sizeof(SimDesc)) != cudaSuccess ||
      cudaMalloc(&E->k, E->nvalues * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&E->dt, n_sims * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&E->smax, n_sims * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&E->err, sizeof(unsigned)) != cudaSuccess) {
    dg_ensemble_destroy(E);
    return fail(DG_ERR_OOM, "dg_ensemble_create: cudaMalloc failed");
  }
  if (cudaMemcpy(E->d_sims, E->sims.data(), n_sims * sizeof(SimDesc), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(E->k, 0, E->nvalues * sizeof(double)) != cudaSuccess ||
      cudaMemset(E->dt, 0, n_sims * sizeof(double)) != cudaSuccess ||
      cudaMemset(E->smax, 0, n_sims * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(E->err, 0, sizeof(unsigned)) != cudaSuccess) {
    dg_ensemble_destroy(E);
    return fail(DG_ERR_CUDA, "dg_ensemble_create: initialisation failed");
  }
  int rc = build_items(E);
  if (rc) {
    dg_ensemble_destroy(E);
    return rc;
  }
  *out = E;
  return DG_OK;
}

int dg_ensemble_info(const dg_ensemble* E, long long* n_values, long long* n_nodes,
                     long long* offsets) {
  if (!E) return fail(DG_ERR_ARG, "dg_ensemble_info: null ensemble");
  if (n_values) *n_values = E->nvalues;
  if (n_nodes) *n_nodes = E->nnodes;
  if (offsets) {
    for (int s = 0; s < E->nsims; ++s) offsets[s] = E->sims[s].off;
    offsets[E->nsims] = E->nvalues;
  }
  return DG_OK;
}

int dg_ensemble_set_dt(dg_ensemble* E, const double* dt_host) {
  if (!E || !dt_host) return fail(DG_ERR_ARG, "dg_ensemble_set_dt: null argument");
  if (cudaMemcpyAsync(E->dt, dt_host, E->nsims * sizeof(double), cudaMemcpyHostToDevice,
                      E->stream) != cudaSuccess ||
      cudaStreamSynchronize(E->stream) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble_set_dt: copy failed");
  return DG_OK;
}

int dg_ensemble_get_dt(dg_ensemble* E, double* dt_host) {
  if (!E || !dt_host) return fail(DG_ERR_ARG, "dg_ensemble_get_dt: null argument");
  if (cudaMemcpyAsync(dt_host, E->dt, E->nsims * sizeof(double), cudaMemcpyDeviceToHost,
                      E->stream) != cudaSuccess ||
      cudaStreamSynchronize(E->stream) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble_get_dt: copy failed");
  return DG_OK;
}

int dg_ensemble_compute_dt(dg_ensemble* E, const double* u, double cfl) {
  if (!E || !u || !(cfl > 0.0)) return fail(DG_ERR_ARG, "dg_ensemble_compute_dt: bad argument");
  return launch_dt(E, u, cfl);
}

int dg_ensemble_stage(dg_ensemble* E, const double* u_in, double* u_out, int stage) {
  if (!E || !u_in || !u_out || u_in == u_out || stage < 0 || stage > 4)
    return fail(DG_ERR_ARG, "dg_ensemble_stage: bad argument (u_in and u_out must differ)");
  return launch_stage(E, u_in, u_out, stage);
}

int dg_ensemble_step(dg_ensemble* E, double* u, double* u_tmp, double cfl) {
  if (!E || !u || !u_tmp || u == u_tmp) return fail(DG_ERR_ARG, "dg_ensemble_step: bad argument");
  return enqueue_step(E, u, u_tmp, cfl);
}

int dg_ensemble_step_graph(dg_ensemble* E, double* u, double* u_tmp, double cfl) {
  if (!E || !u || !u_tmp || u == u_tmp)
    return fail(DG_ERR_ARG, "dg_ensemble_step_graph: bad argument");
  if (!E->graph || E->graph_u != u || E->graph_tmp != u_tmp || E->graph_cfl != cfl) {
    if (E->graph) {
      cudaGraphExecDestroy(E->graph);
      E->graph = nullptr;
    }
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
      return fail(DG_ERR_CUDA, "dg_ensemble_step_graph: stream");
    cudaStream_t saved = E->stream;
    E->stream = cap;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      E->stream = saved;
      cudaStreamDestroy(cap);
      return fail(DG_ERR_CUDA, "dg_ensemble_step_graph: begin capture");
    }
    int rc = enqueue_step(E, u, u_tmp, cfl);
    cudaError_t ce = cudaStreamEndCapture(cap, &g);
    E->stream = saved;
    cudaStreamDestroy(cap);
    if (rc != DG_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc ? rc : fail(DG_ERR_CUDA, "dg_ensemble_step_graph: end capture");
    }
    ce = cudaGraphInstantiate(&E->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(DG_ERR_CUDA, "dg_ensemble_step_graph: instantiate");
    E->graph_u = u;
    E->graph_tmp = u_tmp;
    E->graph_cfl = cfl;
  }
  if (cudaGraphLaunch(E->graph, E->stream) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble_step_graph: launch");
  return DG_OK;
}

int dg_ensemble_rk_reset(dg_ensemble* E) {
  if (!E) return fail(DG_ERR_ARG, "dg_ensemble_rk_reset: null ensemble");
  if (cudaMemsetAsync(E->k, 0, E->nvalues * sizeof(double), E->stream) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble_rk_reset: memset");
  return DG_OK;
}

int dg_ensemble_check(dg_ensemble* E, int* flags) {
  if (!E) return fail(DG_ERR_ARG, "dg_ensemble_check: null ensemble");
  unsigned h = 0;
  if (cudaMemcpyAsync(&h, E->err, sizeof(unsigned), cudaMemcpyDeviceToHost, E->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(E->stream) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble_check: copy");
  if (flags) *flags = (int)h;
  if (h) {
    cudaMemsetAsync(E->err, 0, sizeof(unsigned), E->stream);
    return fail(DG_ERR_NONPHYSICAL, "dg_ensemble: non-physical state met");
  }
  return DG_OK;
}

int dg_ensemble_set_block(dg_ensemble* E, int threads, int blocks_per_sm) {
  if (!E || threads < 32 || threads > 256 || (threads & 31) || blocks_per_sm < 1 ||
      blocks_per_sm > 32)
    return fail(DG_ERR_ARG, "dg_ensemble_set_block: bad configuration");
  for (int N = kEnsMinN; N <= kEnsMaxN; ++N)
    if (items_epb(N, threads) < 1) return fail(DG_ERR_ARG, "dg_ensemble_set_block: CTA too small");
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaStreamSynchronize(E->stream);
  E->block = threads;
  E->grid = nsm * blocks_per_sm;
  if (E->graph) {
    cudaGraphExecDestroy(E->graph);
    E->graph = nullptr;
  }
  return build_items(E);
}

// Autotuner: times one stage for every candidate (threads per CTA, CTAs per
// SM) on (u, u_tmp) and keeps the fastest; the RK register is saved and
// restored around the trials.
int dg_ensemble_tune(dg_ensemble* E, const double* u, double* u_tmp, int* best_threads,
                     int* best_blocks_per_sm, float* best_ms) {
  if (!E || !u || !u_tmp || u == u_tmp) return fail(DG_ERR_ARG, "dg_ensemble_tune: bad argument");
  const int cand_t[] = {64, 128, 192, 256};  // at most the kernel's launch bound
  const int cand_b[] = {2, 4, 8};
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  float best = 1e30f;
  int bt = E->block, bb = E->grid / nsm;
  double* ksave = nullptr;
  if (cudaMalloc(&ksave, E->nvalues * sizeof(double)) != cudaSuccess)
    return fail(DG_ERR_OOM, "dg_ensemble_tune: cudaMalloc");
  cudaMemcpyAsync(ksave, E->k, E->nvalues * sizeof(double), cudaMemcpyDeviceToDevice, E->stream);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int t : cand_t) {
    for (int bp : cand_b) {
      if (dg_ensemble_set_block(E, t, bp) != DG_OK) continue;
      if (launch_stage(E, u, u_tmp, 1) != DG_OK) continue;  // warm-up
      cudaEventRecord(a, E->stream);
      bool ok = true;
      for (int r = 0; r < 3 && ok; ++r) ok = launch_stage(E, u, u_tmp, 1) == DG_OK;
      cudaEventRecord(b, E->stream);
      cudaEventSynchronize(b);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      ms /= 3.0f;
      if (ok && ms < best) {
        best = ms;
        bt = t;
        bb = bp;
      }
    }
  }
  cudaMemcpyAsync(E->k, ksave, E->nvalues * sizeof(double), cudaMemcpyDeviceToDevice, E->stream);
  cudaStreamSynchronize(E->stream);
  cudaFree(ksave);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  int rc = dg_ensemble_set_block(E, bt, bb);
  if (best_threads) *best_threads = bt;
  if (best_blocks_per_sm) *best_blocks_per_sm = bb;
  if (best_ms) *best_ms = best;
  return rc;
}

}  // extern "C"
