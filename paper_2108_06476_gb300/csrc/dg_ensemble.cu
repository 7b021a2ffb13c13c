// Batched ensemble of independent 3D periodic Euler simulations with uneven
// mesh sizes, boxes and polynomial degrees (N in {3, 4, 5}), advanced
// together: one persistent kernel launch per Runge-Kutta stage over a work
// list of (simulation, element batch) items, a graph-capturable step (the
// per-simulation time steps stay on the device) and an autotuner that picks
// the CTA size (hence the elements per work item for every degree) and the
// number of resident CTAs per SM.
//
// A stage launch is cooperative (all its CTAs resident) and runs two phases
// over the work list, separated by a grid-wide barrier:
//   A. for each item: the FP32 references of its elements (FP32 ensembles),
//      then the surface flux of every face node on the right faces of its
//      elements (each face once, by its left element), into the face buffer;
//   B. for each item: the flux-differencing volume term, the lifting of both
//      faces of every line and the stage update k <- A k + dt du,
//      u_out <- u_in + B k.
// Phase B reads only its own elements' states (the faces were read in phase
// A), so u_out may be u_in: a step updates the state in place. The arithmetic
// is that of dg_rhs: the same device functions (face_flux, volume_batch,
// and their FP32 perturbation forms), with each member's own split-form
// tables. The barrier's wait is bounded (about one second); if it runs out,
// the launch sets the timeout bit of the error word and skips phase B, and
// dg_ensemble_check reports DG_ERR_TIMEOUT.
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
void build_tables_fp64(int d, int N, const double* h, Tables<double>* t);
void build_tables_fp32(int d, int N, const double* h, Tables<float>* t);
}

namespace {

using namespace dg;

constexpr int kEnsMinN = 3, kEnsMaxN = 5;
constexpr int kEnsMaxItem = 32;          // elements per work item
constexpr unsigned kErrTimeout = 8u;     // error-word bit: a bounded wait gave up

struct SimDesc {
  int N, n, nelem;
  long long off;     // first value of the member in the state
  long long fsoff;   // first value of the member in the face buffer
  long long refoff;  // first float of the member in the reference buffer
  long long eoff;    // first element of the member (reference energies)
  double lam_scale[3];  // 2/h_k (for the wave-speed sum)
};

struct WorkItem {
  int sim, e0, count;
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
  void* fs;            // face buffer (rhs precision)
  float* ref;          // FP32 references
  double* refE;        // their FP64 energies
  const void* tables;  // per member Tables<R>
  unsigned* err;
  unsigned* bar;       // barrier counter, zero at launch
  int pair;            // FP64: phase B pair-parallel (see ens_volume_pp)
};

int fail(int code, const char* msg) { return dg::set_last_error(code, msg); }

template <int N>
struct EShape {
  static constexpr int NP = N + 1, P = NP * NP * NP, LINES = NP * NP;
};

__device__ __forceinline__ Geom member_geom(const SimDesc& sd, const EnsArgs& a) {
  Geom g;
  g.n[0] = g.n[1] = g.n[2] = sd.n;
  g.nelem = sd.nelem;
  g.gamma = a.gamma;
  g.gm1 = a.gm1;
  g.gm1inv = a.gm1inv;
  return g;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Every CTA of the (cooperative, hence co-resident) launch arrives once;
// returns false for all threads of the CTA if the others did not all arrive
// within about one second (the timeout bit is then set).
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned long long t0 = global_ns();
    int ok = 1;
    while (*(volatile unsigned*)bar < nblocks) {
      if (global_ns() - t0 > 1000000000ull) {
        ok = 0;
        atomicOr(err, kErrTimeout);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// phase A of one item: face fluxes of the right faces of its elements
template <typename R, int N>
__device__ void ens_faces(const EnsArgs& a, const SimDesc& sd, const WorkItem& w) {
  constexpr int LINES = EShape<N>::LINES;
  constexpr bool F32 = sizeof(R) == 4;
  const Geom g = member_geom(sd, a);
  const double* u = a.uin + sd.off;
  R* fs = static_cast<R*>(a.fs) + sd.fsoff;
  float* ref = a.ref + sd.refoff;
  double* refE = a.refE + sd.eoff;
  if (F32) {
    for (int el = threadIdx.x; el < w.count; el += blockDim.x)
      element_ref<3>(u, ref, refE, w.e0 + el, N + 1, a.gm1, a.gm1inv);
    __syncthreads();
  }
  // FP64: the direction is a value, so that warps holding faces of two
  // directions (items of degree 4 and 5) issue one instruction stream (the
  // FP32 face flux, mostly FP32 arithmetic, gained nothing from it)
  const int per_dir = w.count * LINES;
  for (int t = threadIdx.x; t < 3 * per_dir; t += blockDim.x) {
    const int dir = t / per_dir, r = t % per_dir;
    const int e = w.e0 + r / LINES, l = r % LINES;
    if constexpr (F32) {
      if (dir == 0) face_flux32<3, N, 0>(u, (float*)fs, g, a.sf, ref, refE, e, l);
      else if (dir == 1) face_flux32<3, N, 1>(u, (float*)fs, g, a.sf, ref, refE, e, l);
      else face_flux32<3, N, 2>(u, (float*)fs, g, a.sf, ref, refE, e, l);
    } else {
      face_flux_rt<3, N, R>(dir, u, fs, g, a.sf, e, l);
    }
  }
}

// phase B of one item: volume term, lifting and the stage update
template <typename R, int N>
__device__ void ens_volume(const EnsArgs& a, const SimDesc& sd, const WorkItem& w,
                           const Tables<R>& tb, unsigned char* smem) {
  const Geom g = member_geom(sd, a);
  StageFuse fz;
  fz.k = a.k + sd.off;
  fz.dt = a.dt + w.sim;
  fz.a = a.A;
  fz.b = a.B;
  fz.ref = a.ref + sd.refoff;
  fz.refE = a.refE + sd.eoff;
  fz.u_out = a.uout + sd.off;
  double* u = const_cast<double*>(a.uin) + sd.off;
  if constexpr (sizeof(R) == 4)
    volume_batch32<3, N, kVRanocha, kEnsMaxItem>(u, nullptr, static_cast<const float*>(a.fs) + sd.fsoff,
                                                 g, tb, a.err, fz, w.e0, w.count, smem);
  else
    volume_batch<3, N, R, kVRanocha, kEnsMaxItem>(u, nullptr, static_cast<const R*>(a.fs) + sd.fsoff,
                                                  g, tb, a.err, fz, w.e0, w.count, smem);
}

// phase B of one item, pair-parallel (FP64): the item's elements one after
// another, each with the whole CTA: one thread per (line, node pair) of a
// direction evaluates the pair flux into shared memory, then one thread per
// node sums its line in the line-owning order (bitwise the same result)
template <int N>
__device__ void ens_volume_pp(const EnsArgs& a, const SimDesc& sd, const WorkItem& w,
                              const Tables<double>& tb, unsigned char* smem) {
  const Geom g = member_geom(sd, a);
  StageFuse fz;
  fz.k = a.k + sd.off;
  fz.dt = a.dt + w.sim;
  fz.a = a.A;
  fz.b = a.B;
  fz.u_out = a.uout + sd.off;
  double* u = const_cast<double*>(a.uin) + sd.off;
  const double* fs = static_cast<const double*>(a.fs) + sd.fsoff;
  for (int el = 0; el < w.count; ++el)
    pp_elements<3, N, kVRanocha, false, 1, 1, true>(u, nullptr, fs, g, tb, a.err, fz, 0, w.e0 + el, 1,
                                              smem);
}

// one cooperative launch per stage: blocks walk the work list (largest
// degrees first) in each phase; CTAs of at most 128 threads, at least three
// resident per SM (at most 168 registers a thread)
constexpr int kEnsMaxThreads = 128;
template <typename R>
__global__ void __launch_bounds__(kEnsMaxThreads, 3) ensemble_stage_kernel(EnsArgs a) {
  extern __shared__ __align__(16) unsigned char dg_smem[];
  __shared__ Tables<R> s_tb;
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const WorkItem w = a.items[it];
    const SimDesc sd = a.sims[w.sim];
    if (sd.N == 3) ens_faces<R, 3>(a, sd, w);
    else if (sd.N == 4) ens_faces<R, 4>(a, sd, w);
    else ens_faces<R, 5>(a, sd, w);
  }
  if (!grid_barrier(a.bar, gridDim.x, a.err)) return;
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const WorkItem w = a.items[it];
    const SimDesc sd = a.sims[w.sim];
    {
      // the member's coefficients; FP64 members take them times their dt
      // (the fused stage's line sums are then dt du, as in the single-mesh
      // kernel), FP32 members as they are
      const R* src = reinterpret_cast<const R*>(static_cast<const Tables<R>*>(a.tables) + w.sim);
      R* dst = reinterpret_cast<R*>(&s_tb);
      const R sc = sizeof(R) == 8 ? R(a.dt[w.sim]) : R(1);
      for (int i = threadIdx.x; i < (int)(sizeof(Tables<R>) / sizeof(R)); i += blockDim.x)
        dst[i] = sc * src[i];
    }
    __syncthreads();
    if constexpr (sizeof(R) == 8) {
      if (a.pair) {
        if (sd.N == 3) ens_volume_pp<3>(a, sd, w, s_tb, dg_smem);
        else if (sd.N == 4) ens_volume_pp<4>(a, sd, w, s_tb, dg_smem);
        else ens_volume_pp<5>(a, sd, w, s_tb, dg_smem);
        continue;
      }
    }
    if (sd.N == 3) ens_volume<R, 3>(a, sd, w, s_tb, dg_smem);
    else if (sd.N == 4) ens_volume<R, 4>(a, sd, w, s_tb, dg_smem);
    else ens_volume<R, 5>(a, sd, w, s_tb, dg_smem);
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
        const double cs = dg::sqrt_pos(gamma * q.p * rr);
#pragma unroll
        for (int k = 0; k < 3; ++k) lam[k] = fmax(lam[k], fabs(q.v[k]) + cs);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
        for (int off = 16; off > 0; off >>= 1)
          lam[k] = fmax(lam[k], __shfl_xor_sync(0xffffffffu, lam[k], off));
      if (lane == 0) {
        double s = sd.lam_scale[0] * lam[0];
        s = s + sd.lam_scale[1] * lam[1];
        s = s + sd.lam_scale[2] * lam[2];
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

}  // namespace

struct dg_ensemble {
  int nsims;
  dg_options opt;
  cudaStream_t stream;
  std::vector<SimDesc> sims;
  long long nvalues, nnodes, nfs, nref;
  int block;  // threads per CTA (tunable)
  int per_sm; // requested resident CTAs per SM (tunable)
  int pair;   // FP64: pair-parallel volume phase (tunable; 0: one thread per line)
  int grid;   // persistent CTAs (cooperative launch)
  int nitems;
  SimDesc* d_sims;
  WorkItem* d_items;
  void* d_tables;  // per member Tables<R>
  double* k;
  double* dt;
  void* fs;
  float* ref;
  double* refE;
  unsigned long long* smax;
  unsigned* err;
  unsigned* bar;
  cudaGraphExec_t graph;
  const double* graph_u;
  double graph_cfl;
};

namespace {

// elements per work item for degree N with `block` threads per CTA
int items_epb(int N, int block) {
  const int lines = (N + 1) * (N + 1);
  int e = block / lines;
  if (e > kEnsMaxItem) e = kEnsMaxItem;
  return e < 1 ? 0 : e;
}

// dynamic shared memory of a work item: FP64, node slots + accumulators;
// FP32, the same in FP32 plus the staged RK register (volume32_smem);
// pair-parallel, one element's slots, accumulators and pair fluxes of one
// direction
int smem_for(int precision, int block, int pair) {
  if (pair)
    return std::max(PairPar<3, 3, 1>::SMEM,
                    std::max(PairPar<3, 4, 1>::SMEM, PairPar<3, 5, 1>::SMEM));
  int m = 0;
  for (int N = kEnsMinN; N <= kEnsMaxN; ++N) {
    const int P = (N + 1) * (N + 1) * (N + 1), epb = items_epb(N, block);
    const int b = precision == DG_FP64 ? epb * (9 + 5) * P * 8
                                       : ((4 * epb * 14 * P + 15) & ~15) + 8 * epb * 5 * P;
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

template <typename R>
int configure_grid(dg_ensemble* E) {
  const int sm = smem_for(E->opt.precision, E->block, E->pair);
  cudaError_t e = allow_smem(ensemble_stage_kernel<R>, sm);
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, "dg_ensemble: shared-memory attribute");
  int dev = 0, nsm = 0, coop = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return fail(DG_ERR_CUDA, "dg_ensemble: the device has no cooperative launch");
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ensemble_stage_kernel<R>, E->block, sm);
  if (e != cudaSuccess || per < 1) return fail(DG_ERR_CUDA, "dg_ensemble: occupancy query failed");
  // at most the resident CTAs (the barrier needs every CTA of the launch)
  E->grid = nsm * std::min(E->per_sm, per);
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
  a.fs = E->fs;
  a.ref = E->ref;
  a.refE = E->refE;
  a.tables = E->d_tables;
  a.err = E->err;
  a.bar = E->bar;
  a.pair = E->pair;
  if (cudaMemsetAsync(E->bar, 0, sizeof(unsigned), E->stream) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_ensemble: clearing the barrier counter failed");
  const int sm = smem_for(E->opt.precision, E->block, E->pair);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(E->grid);
  cfg.blockDim = dim3(E->block);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = E->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (E->opt.precision == DG_FP64) e = cudaLaunchKernelEx(&cfg, ensemble_stage_kernel<double>, a);
  else e = cudaLaunchKernelEx(&cfg, ensemble_stage_kernel<float>, a);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, cudaGetErrorString(e));
  return DG_OK;
}

int launch_dt(dg_ensemble* E, const double* u, double cfl) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  ensemble_speed_kernel<<<nsm * 4, 256, 0, E->stream>>>(E->d_sims, E->d_items, E->nitems, u,
                                                         E->opt.gamma, E->opt.gamma - 1.0,
                                                         E->smax, E->err);
  ensemble_dt_kernel<<<(E->nsims + 127) / 128, 128, 0, E->stream>>>(E->d_sims, E->nsims, cfl,
                                                                    E->smax, E->dt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, cudaGetErrorString(e));
  return DG_OK;
}

// one step in place on u: (dt from u when cfl > 0), then the five stages
int enqueue_step(dg_ensemble* E, double* u, double cfl) {
  int rc = (cfl > 0.0) ? launch_dt(E, u, cfl) : DG_OK;
  if (rc) return rc;
  for (int s = 0; s < 5; ++s) {
    rc = launch_stage(E, u, u, s);
    if (rc) return rc;
  }
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
  cudaFree(E->d_tables);
  cudaFree(E->k);
  cudaFree(E->dt);
  cudaFree(E->fs);
  cudaFree(E->ref);
  cudaFree(E->refE);
  cudaFree(E->smax);
  cudaFree(E->err);
  cudaFree(E->bar);
  delete E;
  return DG_OK;
}

int dg_ensemble_create(int n_sims, const int* d, const int* N, const int* elements_per_dim,
                       const double* domains, const dg_options* opt, void* cuda_stream,
                       dg_ensemble** out) {
  if (out) *out = nullptr;
  if (!out || !N || !elements_per_dim || n_sims < 1)
    return fail(DG_ERR_ARG, "dg_ensemble_create: bad arguments");
  dg_options o = {1.4, DG_VFLUX_RANOCHA, DG_SFLUX_LLF, DG_FP64};
  if (opt) o = *opt;
  if (!(o.gamma > 1.0) || o.volume_flux != DG_VFLUX_RANOCHA || o.surface_flux < 0 ||
      o.surface_flux > 3 || (o.precision != DG_FP64 && o.precision != DG_FP32))
    return fail(DG_ERR_ARG, "dg_ensemble_create: invalid options (Ranocha volume flux only)");
  for (int s = 0; s < n_sims; ++s) {
    if (d && d[s] != 3) return fail(DG_ERR_ARG, "dg_ensemble_create: members must be 3D (d = 3)");
    if (N[s] < kEnsMinN || N[s] > kEnsMaxN || elements_per_dim[s] < 1 ||
        elements_per_dim[s] > 1024)
      return fail(DG_ERR_ARG, "dg_ensemble_create: N must be in {3,4,5} and 1 <= n <= 1024");
    if (domains)
      for (int k = 0; k < 3; ++k)
        if (!(domains[6 * s + 2 * k + 1] > domains[6 * s + 2 * k]))
          return fail(DG_ERR_ARG, "dg_ensemble_create: every domain needs lo < hi");
  }
  dg_ensemble* E = new dg_ensemble();
  E->nsims = n_sims;
  E->opt = o;
  E->stream = (cudaStream_t)cuda_stream;
  E->block = 128;
  E->per_sm = 4;
  E->pair = 0;
  E->d_sims = nullptr;
  E->d_items = nullptr;
  E->d_tables = nullptr;
  E->k = nullptr;
  E->dt = nullptr;
  E->fs = nullptr;
  E->ref = nullptr;
  E->refE = nullptr;
  E->smax = nullptr;
  E->err = nullptr;
  E->bar = nullptr;
  E->graph = nullptr;
  E->graph_u = nullptr;
  E->graph_cfl = 0.0;
  const size_t rs = o.precision == DG_FP64 ? sizeof(double) : sizeof(float);
  const size_t tsize = o.precision == DG_FP64 ? sizeof(Tables<double>) : sizeof(Tables<float>);
  std::vector<unsigned char> tables(tsize * n_sims);
  long long off = 0, nodes = 0, fsoff = 0, refoff = 0;
  for (int s = 0; s < n_sims; ++s) {
    SimDesc sd;
    sd.N = N[s];
    sd.n = elements_per_dim[s];
    sd.nelem = sd.n * sd.n * sd.n;
    sd.off = off;
    sd.fsoff = fsoff;
    sd.refoff = refoff;
    sd.eoff = refoff / 5;
    double h[3];
    for (int k = 0; k < 3; ++k) {
      const double lo = domains ? domains[6 * s + 2 * k] : -1.0;
      const double hi = domains ? domains[6 * s + 2 * k + 1] : 1.0;
      h[k] = (hi - lo) / sd.n;
      sd.lam_scale[k] = 2.0 / h[k];
    }
    if (o.precision == DG_FP64)
      build_tables_fp64(3, sd.N, h, reinterpret_cast<Tables<double>*>(tables.data()) + s);
    else
      build_tables_fp32(3, sd.N, h, reinterpret_cast<Tables<float>*>(tables.data()) + s);
    const long long P = (long long)(sd.N + 1) * (sd.N + 1) * (sd.N + 1);
    off += 5LL * sd.nelem * P;
    nodes += sd.nelem * P;
    fsoff += 3LL * 5 * sd.nelem * (sd.N + 1) * (sd.N + 1);
    refoff += 5LL * sd.nelem;
    E->sims.push_back(sd);
  }
  E->nvalues = off;
  E->nnodes = nodes;
  E->nfs = fsoff;
  E->nref = refoff;
  if (cudaMalloc(&E->d_sims, n_sims * sizeof(SimDesc)) != cudaSuccess ||
      cudaMalloc(&E->d_tables, tables.size()) != cudaSuccess ||
      cudaMalloc(&E->k, E->nvalues * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&E->dt, n_sims * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&E->fs, E->nfs * rs) != cudaSuccess ||
      cudaMalloc(&E->ref, std::max(E->nref, 1LL) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&E->refE, std::max(E->nref / 5, 1LL) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&E->smax, n_sims * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&E->err, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&E->bar, sizeof(unsigned)) != cudaSuccess) {
    dg_ensemble_destroy(E);
    return fail(DG_ERR_OOM, "dg_ensemble_create: cudaMalloc failed");
  }
  if (cudaMemcpy(E->d_sims, E->sims.data(), n_sims * sizeof(SimDesc), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(E->d_tables, tables.data(), tables.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(E->k, 0, E->nvalues * sizeof(double)) != cudaSuccess ||
      cudaMemset(E->dt, 0, n_sims * sizeof(double)) != cudaSuccess ||
      cudaMemset(E->smax, 0, n_sims * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(E->err, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(E->bar, 0, sizeof(unsigned)) != cudaSuccess) {
    dg_ensemble_destroy(E);
    return fail(DG_ERR_CUDA, "dg_ensemble_create: initialisation failed");
  }
  int rc = build_items(E);
  if (rc == DG_OK)
    rc = (o.precision == DG_FP64) ? configure_grid<double>(E) : configure_grid<float>(E);
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
  if (!E || !u_in || !u_out || stage < 0 || stage > 4)
    return fail(DG_ERR_ARG, "dg_ensemble_stage: bad argument");
  return launch_stage(E, u_in, u_out, stage);
}

int dg_ensemble_step(dg_ensemble* E, double* u, double cfl) {
  if (!E || !u) return fail(DG_ERR_ARG, "dg_ensemble_step: bad argument");
  return enqueue_step(E, u, cfl);
}

int dg_ensemble_step_graph(dg_ensemble* E, double* u, double cfl) {
  if (!E || !u) return fail(DG_ERR_ARG, "dg_ensemble_step_graph: bad argument");
  if (!E->graph || E->graph_u != u || E->graph_cfl != cfl) {
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
    int rc = enqueue_step(E, u, cfl);
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
    if (h & kErrTimeout)
      return fail(DG_ERR_TIMEOUT, "dg_ensemble: a stage's grid barrier timed out");
    return fail(DG_ERR_NONPHYSICAL, "dg_ensemble: non-physical state met");
  }
  return DG_OK;
}

int dg_ensemble_set_block(dg_ensemble* E, int threads, int blocks_per_sm) {
  if (!E || threads < 32 || threads > kEnsMaxThreads || (threads & 31) || blocks_per_sm < 1 ||
      blocks_per_sm > 32)
    return fail(DG_ERR_ARG, "dg_ensemble_set_block: bad configuration");
  for (int N = kEnsMinN; N <= kEnsMaxN; ++N)
    if (items_epb(N, threads) < 1) return fail(DG_ERR_ARG, "dg_ensemble_set_block: CTA too small");
  cudaStreamSynchronize(E->stream);
  E->block = threads;
  E->per_sm = blocks_per_sm;
  if (E->graph) {
    cudaGraphExecDestroy(E->graph);
    E->graph = nullptr;
  }
  int rc = build_items(E);
  if (rc) return rc;
  return (E->opt.precision == DG_FP64) ? configure_grid<double>(E) : configure_grid<float>(E);
}

int dg_ensemble_set_pair_parallel(dg_ensemble* E, int on) {
  if (!E || (on != 0 && on != 1))
    return fail(DG_ERR_ARG, "dg_ensemble_set_pair_parallel: on must be 0 or 1");
  if (on && E->opt.precision != DG_FP64)
    return fail(DG_ERR_ARG, "dg_ensemble_set_pair_parallel: FP64 ensembles only");
  cudaStreamSynchronize(E->stream);
  E->pair = on;
  if (E->graph) {
    cudaGraphExecDestroy(E->graph);
    E->graph = nullptr;
  }
  return (E->opt.precision == DG_FP64) ? configure_grid<double>(E) : configure_grid<float>(E);
}

int dg_ensemble_get_pair_parallel(const dg_ensemble* E, int* on) {
  if (!E || !on) return fail(DG_ERR_ARG, "dg_ensemble_get_pair_parallel: null argument");
  *on = E->pair;
  return DG_OK;
}

int dg_ensemble_get_block(const dg_ensemble* E, int* threads, int* ctas_per_sm, int* grid) {
  if (!E) return fail(DG_ERR_ARG, "dg_ensemble_get_block: null ensemble");
  if (threads) *threads = E->block;
  if (ctas_per_sm) *ctas_per_sm = E->per_sm;
  if (grid) *grid = E->grid;
  return DG_OK;
}

// Autotuner: times one stage for every candidate (threads per CTA, CTAs per
// SM and, for FP64, one thread per line or pair-parallel) from u into u_tmp
// (u is not changed) and keeps the fastest; the RK register is saved and
// restored around the trials.
int dg_ensemble_tune(dg_ensemble* E, const double* u, double* u_tmp, int* best_threads,
                     int* best_blocks_per_sm, float* best_ms) {
  if (!E || !u || !u_tmp || u == u_tmp) return fail(DG_ERR_ARG, "dg_ensemble_tune: bad argument");
  const int cand_t[] = {64, 96, 128};  // at most the kernel's launch bound
  const int cand_b[] = {1, 2, 3, 4, 6};
  float best = 1e30f;
  int bt = E->block, bb = E->per_sm, bp_mode = E->pair;
  const int n_modes = E->opt.precision == DG_FP64 ? 2 : 1;
  double* ksave = nullptr;
  if (cudaMalloc(&ksave, E->nvalues * sizeof(double)) != cudaSuccess)
    return fail(DG_ERR_OOM, "dg_ensemble_tune: cudaMalloc");
  cudaMemcpyAsync(ksave, E->k, E->nvalues * sizeof(double), cudaMemcpyDeviceToDevice, E->stream);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int mode = 0; mode < n_modes; ++mode) {
    if (dg_ensemble_set_pair_parallel(E, mode) != DG_OK) continue;
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
          bp_mode = mode;
        }
      }
    }
  }
  cudaMemcpyAsync(E->k, ksave, E->nvalues * sizeof(double), cudaMemcpyDeviceToDevice, E->stream);
  cudaStreamSynchronize(E->stream);
  cudaFree(ksave);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  int rc = dg_ensemble_set_pair_parallel(E, bp_mode);
  if (rc == DG_OK) rc = dg_ensemble_set_block(E, bt, bb);
  if (best_threads) *best_threads = bt;
  if (best_blocks_per_sm) *best_blocks_per_sm = bb;
  if (best_ms) *best_ms = best;
  return rc;
}

}  // extern "C"
