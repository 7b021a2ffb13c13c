// C ABI of the DGSEM library (declared in include/dgsem.h): mesh set-up with
// the LGL basis (Cartesian, or the warped box with its geometry kernel; Euler
// or 3D ideal MHD), rhs dispatch, the Carpenter-Kennedy stage update and the
// fused steps (device CFL step, given step, CUDA graph, host-resident state),
// the CFL time step, the simulation time and source terms, and the
// compensated integrals.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "dgsem.h"
#include "dg_curved_decl.cuh"
#include "dg_mhd_decl.cuh"
#include "dg_device.cuh"
#include "dg_f32.cuh"

namespace dg {
cudaError_t rhs_launch_double_2(int, const double*, double*, double*, const Geom&,
                                const Tables<double>&, int, int, unsigned*, cudaStream_t, int,
                                const StageFuse&);
cudaError_t rhs_launch_double_3(int, const double*, double*, double*, const Geom&,
                                const Tables<double>&, int, int, unsigned*, cudaStream_t, int,
                                const StageFuse&);
cudaError_t rhs_launch_float_2(int, const double*, float*, float*, const Geom&,
                               const Tables<float>&, int, int, unsigned*, cudaStream_t, int,
                               const StageFuse&);
cudaError_t rhs_launch_float_3(int, const double*, float*, float*, const Geom&,
                               const Tables<float>&, int, int, unsigned*, cudaStream_t, int,
                               const StageFuse&);
cudaError_t vjp_launch_double_2(int, const double*, const double*, double*, double*, const Geom&,
                                const Tables<double>&, int, int, cudaStream_t);
cudaError_t vjp_launch_double_3(int, const double*, const double*, double*, double*, const Geom&,
                                const Tables<double>&, int, int, cudaStream_t);
cudaError_t vjp_launch_float_2(int, const double*, const double*, double*, double*, const Geom&,
                               const Tables<double>&, int, int, cudaStream_t);
cudaError_t vjp_launch_float_3(int, const double*, const double*, double*, double*, const Geom&,
                               const Tables<double>&, int, int, cudaStream_t);
}  // namespace dg

using dg::Geom;
using dg::Tables;

struct dg_mesh {
  int d, N, np, nv;
  int n[3];
  double dom[6];
  double h[3];
  long long nelem, P, nnodes, nvalues;
  dg_options opt;
  cudaStream_t stream;
  Geom geom;
  Tables<double> t64;
  Tables<float> t32;
  double w[dg::kNPMax];
  double* k;           // RK register, nvalues doubles
  void* fs;            // face-flux buffer, d * nv * nelem * (N+1)^(d-1) values
  double* wq;          // quadrature weight of each node of an element, P doubles
  double* partials;    // integral partials, kRedBlocks * 7 * 2 doubles
  double* red_out;     // 7 * 2 doubles
  unsigned long long* speed;  // max wave-speed sum (as ordered bits), then a
                              // block ticket of the fused wave-speed + dt pass
  unsigned* err;       // device error word
  double* fbar;        // face adjoint buffer of dg_rhs_vjp, allocated on first use
  float* ref;          // FP32 meshes: per-element reference states (d+2 floats)
  double* refE;        // FP32 meshes: the references' energies
  double* dt_dev;      // time step computed on the device (dg_step_cfl)
  cudaGraphExec_t graph;
  const double* graph_u;
  double graph_cfl;
  double* u_dev;       // device copy of a host state (dg_step_cfl_host), first use
  double* t_dev;       // simulation time (source terms), advanced by the fused steps
  double* pp_buf;      // small FP64 Cartesian meshes: two stage buffers (2 nvalues)
  // curvilinear meshes (dg_mesh_create_curved)
  int curved;
  double warp;
  int source;          // DG_SOURCE_*
  double* Ja;          // metric terms (J a^r)_n, [e][r][n][P]
  double* invJ;        // 1 / J per node
  double* Jdet;        // J per node
  double* X;           // node coordinates [e][3][P]
  dg::CTables ctab;
  dg::CGeom cgeom;     // curved meshes: the geometry kernel's arguments
  // 3D ideal MHD meshes (dg_mesh_create_mhd)
  int mhd;
  int powell;
  int mhd_sf;           // 0 LLF, 1 HLL, 2 EC
  int mhd_vf;           // 0 weak form, 1 EC flux differencing
  Tables<double> tmhd;  // Ds = -(2/h) D per direction, lifting factors
};

namespace {

thread_local char g_last_error[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define DG_CUDA(call, what)                     \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr int kRedBlocks = 608;  // 4 x 152 SMs
constexpr int kRedThreads = 256;

// ---- LGL basis in long double ----
// Legendre P_n(x) by the three-term recurrence.
long double legendre_p(int n, long double x) {
  if (n == 0) return 1.0L;
  long double a = 1.0L, b = x;
  for (int k = 1; k < n; ++k) {
    long double c = ((2.0L * k + 1.0L) * x * b - k * a) / (k + 1.0L);
    a = b;
    b = c;
  }
  return b;
}

// LGL nodes are the zeros of q(x) = P_{N+1}(x) - P_{N-1}(x) = (2N+1) int P_N,
// with q'(x) = (2N+1) P_N(x); Newton from Chebyshev-Gauss-Lobatto guesses.
// Weights w_j = 2 / (N (N+1) P_N(x_j)^2).
void lgl_basis(int N, long double* x, long double* w) {
  const long double pi = 3.14159265358979323846264338327950288L;
  for (int j = 0; j <= N; ++j) {
    long double t = -cosl(pi * j / N);
    if (j > 0 && j < N) {
      for (int it = 0; it < 200; ++it) {
        long double q = legendre_p(N + 1, t) - legendre_p(N - 1, t);
        long double dq = (2.0L * N + 1.0L) * legendre_p(N, t);
        long double step = q / dq;
        t -= step;
        if (fabsl(step) <= 1e-32L) break;
      }
    }
    x[j] = t;
    long double pn = legendre_p(N, t);
    w[j] = 2.0L / ((long double)N * (N + 1) * pn * pn);
  }
  x[0] = -1.0L;
  x[N] = 1.0L;
}

// Split-form matrix Dt = 2 D - W^-1 B from the closed-form LGL
// differentiation matrix D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) (i != j),
// D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0.
void split_matrix(int N, const long double* x, const long double* w, long double Dt[8][8]) {
  for (int i = 0; i <= N; ++i) {
    for (int j = 0; j <= N; ++j) {
      long double dij;
      if (i != j) dij = legendre_p(N, x[i]) / (legendre_p(N, x[j]) * (x[i] - x[j]));
      else if (i == 0) dij = -(long double)N * (N + 1) / 4.0L;
      else if (i == N) dij = (long double)N * (N + 1) / 4.0L;
      else dij = 0.0L;
      long double b = (i == j && i == 0) ? -1.0L : (i == j && i == N) ? 1.0L : 0.0L;
      Dt[i][j] = 2.0L * dij - b / w[i];
    }
  }
}

// the LGL differentiation matrix itself (same closed form)
void diff_matrix(int N, const long double* x, long double D[8][8]) {
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) {
      if (i != j) D[i][j] = legendre_p(N, x[i]) / (legendre_p(N, x[j]) * (x[i] - x[j]));
      else if (i == 0) D[i][j] = -(long double)N * (N + 1) / 4.0L;
      else if (i == N) D[i][j] = (long double)N * (N + 1) / 4.0L;
      else D[i][j] = 0.0L;
    }
}

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage scheme
// (A, B; the stage times c_s, used by time-dependent source terms, follow).
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0,
                        -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0,
                        -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};
const double kRkC[5] = {0.0, 1432997174477.0 / 9575080441755.0,
                        2526269341429.0 / 6820363962896.0,
                        2006345519317.0 / 3224310063776.0,
                        2802321613138.0 / 2924317926251.0};

// ---- kernels ----
template <typename RD>
__global__ void rk_stage_kernel(double* __restrict__ u, double* __restrict__ k,
                                const RD* __restrict__ du, double a, double b, double dt,
                                long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long n2 = n / 2;
  double2* u2 = reinterpret_cast<double2*>(u);
  double2* k2 = reinterpret_cast<double2*>(k);
  // k <- a k + dt du as fma(a, k, dt du); a = 0 (the first stage) reads no k
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    double2 kk, uu = u2[i];
    double d0, d1;
    if (sizeof(RD) == 8) {
      const double2 dd = reinterpret_cast<const double2*>(du)[i];
      d0 = dd.x;
      d1 = dd.y;
    } else {
      const float2 dd = reinterpret_cast<const float2*>(du)[i];
      d0 = dd.x;
      d1 = dd.y;
    }
    kk.x = dt * d0;
    kk.y = dt * d1;
    if (a != 0.0) {
      const double2 k0 = k2[i];
      kk.x = fma(a, k0.x, kk.x);
      kk.y = fma(a, k0.y, kk.y);
    }
    uu.x = uu.x + b * kk.x;
    uu.y = uu.y + b * kk.y;
    k2[i] = kk;
    u2[i] = uu;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
    const long long i = n - 1;
    double kk = dt * (double)du[i];
    if (a != 0.0) kk = fma(a, k[i], kk);
    k[i] = kk;
    u[i] = u[i] + b * kk;
  }
}

// Max over elements of sum_k (2/h_k) max_nodes(|v_k| + c); one warp per
// element, one atomic per block on the ordered bit pattern of the result.
// R = float evaluates the wave speeds in FP32 (FP32 meshes: the time step
// needs no more than a few digits), R = double as the FP64 path.
__device__ __forceinline__ void speed_node(const double* c, int D, const Geom& g, double* lam,
                                           unsigned& bad, double) {
  double cc[5];
  for (int v = 0; v < D + 2; ++v) cc[v] = c[v];
  double rr;
  if (D == 2) {
    const dg::Prim<double, 2> q = dg::prim_rcp<2>(cc, g.gm1, rr);
    bad |= dg::prim_check(q);
    const double cs = dg::sqrt_pos(g.gamma * q.p * rr);
    for (int k = 0; k < 2; ++k) lam[k] = dg::fmax_nn(lam[k], fabs(q.v[k]) + cs);
  } else {
    const dg::Prim<double, 3> q = dg::prim_rcp<3>(cc, g.gm1, rr);
    bad |= dg::prim_check(q);
    const double cs = dg::sqrt_pos(g.gamma * q.p * rr);
    for (int k = 0; k < 3; ++k) lam[k] = dg::fmax_nn(lam[k], fabs(q.v[k]) + cs);
  }
}
// (FP32: the maxima stay in float and the state is converted on the integer
// pipe, d2f, so that no FP64-pipe instruction runs per node)
__device__ __forceinline__ void speed_node(const double* c, int D, const Geom& g, float* lam,
                                           unsigned& bad, float) {
  const float rho = dg::d2f(c[0]);
  const float rr = 1.0f / rho;
  float v[3], v2 = 0.0f;
  for (int k = 0; k < D; ++k) {
    v[k] = dg::d2f(c[1 + k]) * rr;
    v2 = fmaf(v[k], v[k], v2);
  }
  const float p = (float)g.gm1 * (dg::d2f(c[D + 1]) - 0.5f * rho * v2);
  if (!(rho > 0.0f)) bad |= dg::kErrRho;
  if (!(p > 0.0f)) bad |= dg::kErrP;
  if (!isfinite(rho) || !isfinite(p)) bad |= dg::kErrNaN;
  const float cs = sqrtf((float)g.gamma * p * rr);
  for (int k = 0; k < D; ++k) lam[k] = fmaxf(lam[k], fabsf(v[k]) + cs);
}

// copy_to (optional) receives a copy of u: the host-state step reads a
// mapped host buffer here once and continues on the device copy. dt
// (optional): the last block to finish (a ticket in out[1]) also computes
// dt = cfl 2 / ((N+1) worst) and clears out[0] and out[1], as dt_kernel does.
// epw elements per warp (32 / P when P is 4, 8 or 16, else 1): each element
// takes a segment of 32 / epw lanes, so that FP64 work fills the warps
template <int D, typename R>
__global__ void speed_kernel(const double* __restrict__ u, Geom g, int P, int epw, double s0,
                             double s1, double s2, unsigned long long* out, unsigned* err,
                             double* __restrict__ copy_to, int N, double cfl, double* dt) {
  constexpr int NV = D + 2;
  const int lane = threadIdx.x & 31;
  const int seg = 32 / epw, sub = lane / seg;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double best = 0.0;
  unsigned bad = 0;
  for (long long eb = warp * epw; eb < g.nelem; eb += nwarps * epw) {
    const long long e = eb + sub;
    R lamr[3] = {R(0), R(0), R(0)};
    for (int node = lane % seg; node < P && e < g.nelem; node += seg) {
      double c[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) c[v] = u[(e * NV + v) * P + node];
      if (copy_to) {
#pragma unroll
        for (int v = 0; v < NV; ++v) copy_to[(e * NV + v) * P + node] = c[v];
      }
      speed_node(c, D, g, lamr, bad, R(0));
    }
    double lam[3];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      lam[k] = (double)lamr[k];
      for (int off = seg / 2; off > 0; off >>= 1)
        lam[k] = fmax(lam[k], __shfl_xor_sync(0xffffffffu, lam[k], off));
    }
    double s = s0 * lam[0];
    s = s + s1 * lam[1];
    if (D == 3) s = s + s2 * lam[2];
    best = fmax(best, s);
  }
  __shared__ double sb[32];
  if (lane == 0) sb[threadIdx.x >> 5] = best;
  if (bad) atomicOr(err, bad);
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sb[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
    if (dt) {
      __threadfence();
      if (atomicAdd(out + 1, 1ull) == (unsigned long long)gridDim.x - 1ull) {
        // every block's maximum is in
        const double worst = __longlong_as_double((long long)atomicAdd(out, 0ull));
        out[0] = 0ull;
        out[1] = 0ull;
        if (!(worst > 0.0)) {
          atomicOr(err, 4u);
          *dt = 0.0;
        } else {
          *dt = cfl * 2.0 / ((N + 1) * worst);
        }
      }
    }
  }
}

// dt = cfl 2 / ((N+1) worst) on the device from the wave-speed word, which is
// cleared for the next reduction
__global__ void dt_kernel(unsigned long long* speed, int N, double cfl, double* dt,
                          unsigned* err) {
  const double worst = __longlong_as_double((long long)*speed);
  *speed = 0ull;
  if (!(worst > 0.0)) {
    atomicOr(err, 4u);
    *dt = 0.0;
    return;
  }
  *dt = cfl * 2.0 / ((N + 1) * worst);
}

// a given time step; the simulation time advanced by the step's dt
__global__ void set_dt_kernel(double* dt_dev, double dt) { *dt_dev = dt; }
__global__ void advance_time_kernel(double* t, const double* dt) { *t += *dt; }

// double-double accumulation (Knuth two-sum)
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const double s = a.hi + b.hi;
  const double bb = s - a.hi;
  const double err = (a.hi - (s - bb)) + (b.hi - bb);
  const double lo = a.lo + b.lo + err;
  const double hi = s + lo;
  return dd{hi, lo - (hi - s)};
}
__device__ __forceinline__ dd dd_add1(dd a, double x) { return dd_add(a, dd{x, 0.0}); }

template <int D>
__global__ void integrals_kernel(const double* __restrict__ u, Geom g, int P,
                                 const double* __restrict__ wq, const double* __restrict__ Jn,
                                 double* __restrict__ partials, unsigned* err) {
  constexpr int NV = D + 2, NQ = D + 4;
  dd acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = dd{0.0, 0.0};
  const long long total = g.nelem * P;
  const double gm1 = g.gamma - 1.0;
  unsigned bad = 0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / P;
    const int node = (int)(t % P);
    double c[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) c[v] = u[(e * NV + v) * P + node];
    const dg::Prim<double, D> q = dg::cons2prim<double, D>(c, gm1);
    bad |= dg::prim_check(q);
    const double w = Jn ? wq[node] * Jn[t] : wq[node];  // curved meshes: w J
    double v2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) v2 += q.v[k] * q.v[k];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = dd_add1(acc[v], w * c[v]);
    acc[NV] = dd_add1(acc[NV], w * (-q.rho * (log(q.p) - g.gamma * log(q.rho)) / gm1));
    acc[NV + 1] = dd_add1(acc[NV + 1], w * (0.5 * q.rho * v2));
  }
  if (bad) atomicOr(err, bad);
  __shared__ double sh[kRedThreads][2];
  for (int q = 0; q < NQ; ++q) {
    sh[threadIdx.x][0] = acc[q].hi;
    sh[threadIdx.x][1] = acc[q].lo;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) {
        dd r = dd_add(dd{sh[threadIdx.x][0], sh[threadIdx.x][1]},
                      dd{sh[threadIdx.x + s][0], sh[threadIdx.x + s][1]});
        sh[threadIdx.x][0] = r.hi;
        sh[threadIdx.x][1] = r.lo;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      partials[(blockIdx.x * 7 + q) * 2 + 0] = sh[0][0];
      partials[(blockIdx.x * 7 + q) * 2 + 1] = sh[0][1];
    }
    __syncthreads();
  }
}

__global__ void integrals_final_kernel(const double* __restrict__ partials, int nblocks, int nq,
                                       double* __restrict__ out) {
  __shared__ double sh[kRedThreads][2];
  for (int q = 0; q < nq; ++q) {
    dd a{0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
      a = dd_add(a, dd{partials[(b * 7 + q) * 2], partials[(b * 7 + q) * 2 + 1]});
    sh[threadIdx.x][0] = a.hi;
    sh[threadIdx.x][1] = a.lo;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) {
        dd r = dd_add(dd{sh[threadIdx.x][0], sh[threadIdx.x][1]},
                      dd{sh[threadIdx.x + s][0], sh[threadIdx.x + s][1]});
        sh[threadIdx.x][0] = r.hi;
        sh[threadIdx.x][1] = r.lo;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[2 * q] = sh[0][0];
      out[2 * q + 1] = sh[0][1];
    }
    __syncthreads();
  }
}

bool valid_mesh(const dg_mesh* m) { return m != nullptr && m->k != nullptr; }

int grid_for(long long work, int threads);

// wave-speed reduction into m->speed (FP32 arithmetic on FP32 meshes);
// copy_to (optional): device buffer that receives a copy of u; cfl > 0 on
// Cartesian Euler meshes: the same launch writes the time step to m->dt_dev
// (*dt_done is then set)
int launch_speed(dg_mesh* m, const double* u, double* copy_to = nullptr, double cfl = 0.0,
                 bool* dt_done = nullptr) {
  if (dt_done) *dt_done = false;
  // one warp per element; small meshes get one-warp blocks so that the FP64
  // work (2 lanes per clock per SM) spreads over more SMs
  const int threads = (m->nelem * 32 < 152LL * 4 * 256) ? 32 : 256;
  int grid = grid_for(m->nelem * 32, threads);
  if (m->mhd && m->curved) {
    DG_CUDA(dg::mhd_curved_speed_launch(u, m->Ja, m->invJ, m->geom, (int)m->P, m->speed, m->err,
                                        copy_to, grid, threads, m->stream),
            "MHD curved speed kernel launch");
    return DG_OK;
  }
  if (m->mhd) {
    const double s[3] = {2.0 / m->h[0], 2.0 / m->h[1], 2.0 / m->h[2]};
    DG_CUDA(dg::mhd_speed_launch(u, m->geom, (int)m->P, s, m->speed, m->err, copy_to, grid,
                                 threads, m->stream),
            "MHD speed kernel launch");
    return DG_OK;
  }
  if (m->curved) {
    DG_CUDA(dg::curved_speed_launch(m->N, u, m->Ja, m->invJ, m->geom, m->speed, m->err, copy_to,
                                    grid, threads, m->stream),
            "curved speed kernel launch");
    return DG_OK;
  }
  const double s0 = 2.0 / m->h[0], s1 = 2.0 / m->h[1], s2 = 2.0 / m->h[2];
  const bool f32 = m->opt.precision == DG_FP32;
  double* dt = cfl > 0.0 ? m->dt_dev : nullptr;
  const int P = (int)m->P;
  const int epw = (P == 4 || P == 8 || P == 16) ? 32 / P : 1;
  if (epw > 1) grid = grid_for((m->nelem + epw - 1) / epw * 32, threads);
  if (m->d == 2) {
    if (f32)
      speed_kernel<2, float><<<grid, threads, 0, m->stream>>>(u, m->geom, P, epw, s0, s1, s2,
                                                              m->speed, m->err, copy_to, m->N,
                                                              cfl, dt);
    else
      speed_kernel<2, double><<<grid, threads, 0, m->stream>>>(u, m->geom, P, epw, s0, s1, s2,
                                                               m->speed, m->err, copy_to, m->N,
                                                               cfl, dt);
  } else {
    if (f32)
      speed_kernel<3, float><<<grid, threads, 0, m->stream>>>(u, m->geom, P, epw, s0, s1, s2,
                                                              m->speed, m->err, copy_to, m->N,
                                                              cfl, dt);
    else
      speed_kernel<3, double><<<grid, threads, 0, m->stream>>>(u, m->geom, P, epw, s0, s1, s2,
                                                               m->speed, m->err, copy_to, m->N,
                                                               cfl, dt);
  }
  DG_CUDA(cudaGetLastError(), "speed kernel launch");
  if (dt_done) *dt_done = dt != nullptr;
  return DG_OK;
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

namespace dg {
// Internal helpers for other translation units of the library (not exported
// in the C header): record a failure message, and build the FP64 split-form
// tables of a uniform mesh with element widths h[0..d-1].
int set_last_error(int code, const char* msg) { return fail(code, "%s", msg); }

void build_tables_fp64(int d, int N, const double* h, Tables<double>* t) {
  long double x[8], w[8], Dt[8][8];
  lgl_basis(N, x, w);
  split_matrix(N, x, w, Dt);
  memset(t, 0, sizeof(*t));
  for (int k = 0; k < d; ++k) {
    const long double s = -2.0L / (long double)h[k];
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N; ++b) t->Ds[k][a][b] = (double)(s * Dt[a][b]);
    t->liftR[k] = (double)(s / w[N]);
    t->liftL[k] = (double)(-s / w[0]);
  }
}

// the same tables rounded from long double to FP32
void build_tables_fp32(int d, int N, const double* h, Tables<float>* t) {
  long double x[8], w[8], Dt[8][8];
  lgl_basis(N, x, w);
  split_matrix(N, x, w, Dt);
  memset(t, 0, sizeof(*t));
  for (int k = 0; k < d; ++k) {
    const long double s = -2.0L / (long double)h[k];
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N; ++b) t->Ds[k][a][b] = (float)(s * Dt[a][b]);
    t->liftR[k] = (float)(s / w[N]);
    t->liftL[k] = (float)(-s / w[0]);
  }
}
}  // namespace dg

extern "C" {

const char* dg_last_error(void) { return g_last_error; }

int dg_lgl_nodes(int N, double* xi, double* w) {
  if (N < 1 || N > 7 || !xi || !w) return fail(DG_ERR_ARG, "dg_lgl_nodes: N must be in [1, 7]");
  long double x[8], ww[8];
  lgl_basis(N, x, ww);
  for (int j = 0; j <= N; ++j) {
    xi[j] = (double)x[j];
    w[j] = (double)ww[j];
  }
  return DG_OK;
}

int dg_mesh_create(int d, int N, const int* epd, const double* domain, const dg_options* opt,
                   void* cuda_stream, dg_mesh** out) {
  if (out) *out = nullptr;
  if (!out || !epd || !domain) return fail(DG_ERR_ARG, "dg_mesh_create: null argument");
  if (d < 2 || d > 3) return fail(DG_ERR_ARG, "dg_mesh_create: d must be 2 or 3 (got %d)", d);
  if (N < 1 || N > 7) return fail(DG_ERR_ARG, "dg_mesh_create: N must be in [1, 7] (got %d)", N);
  dg_options o = {1.4, DG_VFLUX_RANOCHA, DG_SFLUX_LLF, DG_FP64};
  if (opt) o = *opt;
  if (!(o.gamma > 1.0) || o.volume_flux < 0 || o.volume_flux > 2 || o.surface_flux < 0 ||
      o.surface_flux > 3 || (o.precision != DG_FP64 && o.precision != DG_FP32))
    return fail(DG_ERR_ARG, "dg_mesh_create: invalid options");
  dg_mesh* m = new dg_mesh();
  memset(m, 0, sizeof(*m));
  m->d = d;
  m->N = N;
  m->np = N + 1;
  m->nv = d + 2;
  m->opt = o;
  m->stream = (cudaStream_t)cuda_stream;
  m->nelem = 1;
  m->P = 1;
  for (int k = 0; k < 3; ++k) {
    m->n[k] = 1;
    m->h[k] = 1.0;
  }
  for (int k = 0; k < d; ++k) {
    if (epd[k] < 1 || !(domain[2 * k + 1] > domain[2 * k])) {
      delete m;
      return fail(DG_ERR_ARG, "dg_mesh_create: bad elements_per_dim or domain in direction %d", k);
    }
    m->n[k] = epd[k];
    m->dom[2 * k] = domain[2 * k];
    m->dom[2 * k + 1] = domain[2 * k + 1];
    m->h[k] = (domain[2 * k + 1] - domain[2 * k]) / epd[k];
    m->nelem *= epd[k];
    m->P *= m->np;
  }
  if (m->nelem > (1LL << 31)) {
    delete m;
    return fail(DG_ERR_ARG, "dg_mesh_create: too many elements");
  }
  m->nnodes = m->nelem * m->P;
  m->nvalues = m->nnodes * m->nv;
  m->geom.n[0] = m->n[0];
  m->geom.n[1] = m->n[1];
  m->geom.n[2] = m->n[2];
  m->geom.nelem = m->nelem;
  m->geom.gamma = o.gamma;
  m->geom.gm1 = o.gamma - 1.0;
  m->geom.gm1inv = 1.0 / (o.gamma - 1.0);

  // basis and scaled split-form tables
  long double x[8], w[8], Dt[8][8];
  lgl_basis(N, x, w);
  split_matrix(N, x, w, Dt);
  memset(&m->t64, 0, sizeof(m->t64));
  memset(&m->t32, 0, sizeof(m->t32));
  for (int k = 0; k < d; ++k) {
    const long double s = -2.0L / (long double)m->h[k];
    for (int a = 0; a <= N; ++a)
      for (int b = 0; b <= N; ++b) {
        m->t64.Ds[k][a][b] = (double)(s * Dt[a][b]);
        m->t32.Ds[k][a][b] = (float)(s * Dt[a][b]);
      }
    m->t64.liftR[k] = (double)(s / w[N]);
    m->t64.liftL[k] = (double)(-s / w[0]);
    m->t32.liftR[k] = (float)(s / w[N]);
    m->t32.liftL[k] = (float)(-s / w[0]);
  }
  for (int j = 0; j <= N; ++j) m->w[j] = (double)w[j];

  // node quadrature weights jac * w_i * w_j (* w_k)
  double jac = 1.0;
  for (int k = 0; k < d; ++k) jac *= 0.5 * m->h[k];
  double wq_host[512];
  for (long long node = 0; node < m->P; ++node) {
    double wqv = jac;
    long long r = node;
    for (int k = 0; k < d; ++k) {
      wqv *= m->w[r % m->np];
      r /= m->np;
    }
    wq_host[node] = wqv;
  }

  const size_t rsize = (o.precision == DG_FP64) ? sizeof(double) : sizeof(float);
  const long long nfaces_vals = (long long)d * m->nv * m->nelem * (m->P / m->np);
  cudaError_t e;
  if ((e = cudaMalloc(&m->k, m->nvalues * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->fs, nfaces_vals * rsize)) != cudaSuccess ||
      (e = cudaMalloc(&m->wq, m->P * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->partials, kRedBlocks * 7 * 2 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->red_out, 7 * 2 * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->speed, 2 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&m->err, sizeof(unsigned))) != cudaSuccess ||
      (e = cudaMalloc(&m->ref, m->nelem * m->nv * sizeof(float))) != cudaSuccess ||
      (e = cudaMalloc(&m->refE, m->nelem * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->dt_dev, sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->t_dev, sizeof(double))) != cudaSuccess ||
      (o.precision == DG_FP64 && m->nelem < dg::kPairParallelElems &&
       (e = cudaMalloc(&m->pp_buf, 2 * m->nvalues * sizeof(double))) != cudaSuccess)) {
    int rc = cuda_fail(e, "dg_mesh_create: cudaMalloc");
    cudaFree(m->k);
    cudaFree(m->fs);
    cudaFree(m->wq);
    cudaFree(m->partials);
    cudaFree(m->red_out);
    cudaFree(m->speed);
    cudaFree(m->err);
    cudaFree(m->ref);
    cudaFree(m->refE);
    cudaFree(m->dt_dev);
    cudaFree(m->t_dev);
    cudaFree(m->pp_buf);
    delete m;
    return rc;
  }
  if ((e = cudaMemcpyAsync(m->wq, wq_host, m->P * sizeof(double), cudaMemcpyHostToDevice,
                           m->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(m->k, 0, m->nvalues * sizeof(double), m->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(m->err, 0, sizeof(unsigned), m->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(m->speed, 0, 2 * sizeof(unsigned long long), m->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(m->dt_dev, 0, sizeof(double), m->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(m->t_dev, 0, sizeof(double), m->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
    int rc = cuda_fail(e, "dg_mesh_create: initialisation");
    dg_mesh_destroy(m);
    return rc;
  }
  *out = m;
  return DG_OK;
}

int dg_mesh_create_curved(int N, const int* epd, double warp, const dg_options* opt,
                          void* cuda_stream, dg_mesh** out) {
  if (out) *out = nullptr;
  if (!out || !epd) return fail(DG_ERR_ARG, "dg_mesh_create_curved: null argument");
  if (!isfinite(warp) || fabs(warp) > 0.5)
    return fail(DG_ERR_ARG, "dg_mesh_create_curved: warp must be finite and |warp| <= 0.5");
  if (opt && opt->precision != DG_FP64)
    return fail(DG_ERR_ARG, "dg_mesh_create_curved: curved meshes are FP64");
  const double box[6] = {-1.0, 1.0, -1.0, 1.0, -1.0, 1.0};
  dg_mesh* m = nullptr;
  int rc = dg_mesh_create(3, N, epd, box, opt, cuda_stream, &m);
  if (rc != DG_OK) return rc;
  m->curved = 1;
  m->warp = warp;
  const long long nn = m->nnodes;
  cudaError_t e;
  if ((e = cudaMalloc(&m->Ja, 9 * nn * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->invJ, nn * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->Jdet, nn * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->X, 3 * nn * sizeof(double))) != cudaSuccess) {
    rc = cuda_fail(e, "dg_mesh_create_curved: cudaMalloc");
    dg_mesh_destroy(m);
    return rc;
  }
  // basis: nodes, derivative matrix, unscaled split form with the sign of du
  long double x[8], w[8], D[8][8], Dt[8][8];
  lgl_basis(N, x, w);
  diff_matrix(N, x, D);
  split_matrix(N, x, w, Dt);
  dg::CGeom cg;
  memset(&cg, 0, sizeof(cg));
  cg.g = m->geom;
  cg.warp = warp;
  memset(&m->ctab, 0, sizeof(m->ctab));
  for (int a = 0; a <= N; ++a) {
    cg.xi[a] = (double)x[a];
    for (int b = 0; b <= N; ++b) {
      cg.D[a][b] = (double)D[a][b];
      m->ctab.Ds[a][b] = (double)(-Dt[a][b]);
    }
  }
  m->ctab.liftR = (double)(-1.0L / w[N]);
  m->ctab.liftL = (double)(1.0L / w[0]);
  cg.Xin = nullptr;
  m->cgeom = cg;
  // reference quadrature weights (the integrals multiply by J per node)
  double wq_host[512];
  for (long long node = 0; node < m->P; ++node)
    wq_host[node] = m->w[node % m->np] * m->w[(node / m->np) % m->np] * m->w[node / (m->np * m->np)];
  if ((e = dg::curved_geometry_launch(N, cg, m->Ja, m->invJ, m->Jdet, m->X, m->stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(m->wq, wq_host, m->P * sizeof(double), cudaMemcpyHostToDevice,
                           m->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
    rc = cuda_fail(e, "dg_mesh_create_curved: geometry");
    dg_mesh_destroy(m);
    return rc;
  }
  *out = m;
  return DG_OK;
}

namespace {
__global__ void reciprocal_kernel(const double* __restrict__ J, double* __restrict__ invJ,
                                  long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    invJ[i] = 1.0 / J[i];
}
}  // namespace

int dg_mesh_set_metric(dg_mesh* m, const double* Ja, const double* J) {
  if (!valid_mesh(m) || !Ja || !J) return fail(DG_ERR_ARG, "dg_mesh_set_metric: null argument");
  if (!m->curved) return fail(DG_ERR_ARG, "dg_mesh_set_metric: not a curved mesh");
  const long long nn = m->nnodes;
  DG_CUDA(cudaMemcpyAsync(m->Ja, Ja, 9 * nn * sizeof(double), cudaMemcpyDeviceToDevice, m->stream),
          "dg_mesh_set_metric: copy");
  DG_CUDA(cudaMemcpyAsync(m->Jdet, J, nn * sizeof(double), cudaMemcpyDeviceToDevice, m->stream),
          "dg_mesh_set_metric: copy");
  reciprocal_kernel<<<grid_for(nn, 256), 256, 0, m->stream>>>(m->Jdet, m->invJ, nn);
  DG_CUDA(cudaGetLastError(), "dg_mesh_set_metric: launch");
  return DG_OK;
}

int dg_mesh_set_nodes(dg_mesh* m, const double* X) {
  if (!valid_mesh(m) || !X) return fail(DG_ERR_ARG, "dg_mesh_set_nodes: null argument");
  if (!m->curved) return fail(DG_ERR_ARG, "dg_mesh_set_nodes: not a curved mesh");
  if ((reinterpret_cast<uintptr_t>(X) & 7) != 0)
    return fail(DG_ERR_ARG, "dg_mesh_set_nodes: X must be 8-byte aligned");
  dg::CGeom cg = m->cgeom;
  cg.Xin = X;
  DG_CUDA(dg::curved_geometry_launch(m->N, cg, m->Ja, m->invJ, m->Jdet, m->X, m->stream),
          "dg_mesh_set_nodes: geometry");
  return DG_OK;
}

namespace {
// Check and translate the MHD options; *euler receives options that the Euler
// creators accept (the MHD path reads its own flux ids).
int mhd_options(const char* who, const dg_options* opt, int powell, dg_options* euler, int* vf,
                int* sf) {
  dg_options o = {5.0 / 3.0, DG_VFLUX_CENTRAL, DG_SFLUX_LLF, DG_FP64};
  if (opt) o = *opt;
  if (!(o.gamma > 1.0) || (powell != 0 && powell != 1) ||
      (o.volume_flux != DG_VFLUX_CENTRAL && o.volume_flux != DG_VFLUX_EC) ||
      (o.surface_flux != DG_SFLUX_LLF && o.surface_flux != DG_SFLUX_HLL &&
       o.surface_flux != DG_SFLUX_EC) ||
      o.precision != DG_FP64)
    return fail(DG_ERR_ARG,
                "%s: needs gamma > 1, powell 0 or 1, the central or EC volume flux, an LLF, HLL "
                "or EC surface flux and FP64",
                who);
  *vf = o.volume_flux == DG_VFLUX_EC ? 1 : 0;
  *sf = o.surface_flux == DG_SFLUX_HLL ? 1 : (o.surface_flux == DG_SFLUX_EC ? 2 : 0);
  o.volume_flux = DG_VFLUX_CENTRAL;
  o.surface_flux = DG_SFLUX_LLF;
  *euler = o;
  return DG_OK;
}

// Turn a freshly created 3D mesh into an MHD mesh: eight variables (the RK
// register and the face buffer, nine values per face node, sized anew) and
// the weak-form tables Ds = -(2/h) D. Destroys the mesh on failure.
int make_mhd(dg_mesh* m, int vf, int sf, int powell, const char* who) {
  m->mhd = 1;
  m->mhd_sf = sf;
  m->mhd_vf = vf;
  m->powell = powell;
  cudaFree(m->k);
  cudaFree(m->fs);
  m->k = nullptr;
  m->fs = nullptr;
  m->nv = 8;
  m->nvalues = m->nnodes * 8;
  const long long nface = 3LL * 9 * m->nelem * (m->P / m->np);
  cudaError_t e;
  if ((e = cudaMalloc(&m->k, m->nvalues * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&m->fs, nface * sizeof(double))) != cudaSuccess ||
      (e = cudaMemsetAsync(m->k, 0, m->nvalues * sizeof(double), m->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(m->stream)) != cudaSuccess) {
    const int rc = cuda_fail(e, who);
    dg_mesh_destroy(m);
    return rc;
  }
  long double x[8], w[8], D[8][8];
  lgl_basis(m->N, x, w);
  diff_matrix(m->N, x, D);
  memset(&m->tmhd, 0, sizeof(m->tmhd));
  for (int k = 0; k < 3; ++k) {
    const long double sc = -2.0L / (long double)m->h[k];
    for (int a = 0; a <= m->N; ++a)
      for (int b = 0; b <= m->N; ++b) m->tmhd.Ds[k][a][b] = (double)(sc * D[a][b]);
    m->tmhd.liftR[k] = (double)(sc / w[m->N]);
    m->tmhd.liftL[k] = (double)(-sc / w[0]);
  }
  return DG_OK;
}
}  // namespace

int dg_mesh_create_mhd(int N, const int* epd, const double* domain, const dg_options* opt,
                       int powell, void* cuda_stream, dg_mesh** out) {
  if (out) *out = nullptr;
  if (!out || !epd || !domain) return fail(DG_ERR_ARG, "dg_mesh_create_mhd: null argument");
  dg_options o;
  int vf, sf;
  int rc = mhd_options("dg_mesh_create_mhd", opt, powell, &o, &vf, &sf);
  if (rc != DG_OK) return rc;
  dg_mesh* m = nullptr;
  if ((rc = dg_mesh_create(3, N, epd, domain, &o, cuda_stream, &m)) != DG_OK) return rc;
  if ((rc = make_mhd(m, vf, sf, powell, "dg_mesh_create_mhd: cudaMalloc")) != DG_OK) return rc;
  *out = m;
  return DG_OK;
}

int dg_mesh_create_mhd_curved(int N, const int* epd, double warp, const dg_options* opt,
                              int powell, void* cuda_stream, dg_mesh** out) {
  if (out) *out = nullptr;
  if (!out || !epd) return fail(DG_ERR_ARG, "dg_mesh_create_mhd_curved: null argument");
  dg_options o;
  int vf, sf;
  int rc = mhd_options("dg_mesh_create_mhd_curved", opt, powell, &o, &vf, &sf);
  if (rc != DG_OK) return rc;
  dg_mesh* m = nullptr;
  if ((rc = dg_mesh_create_curved(N, epd, warp, &o, cuda_stream, &m)) != DG_OK) return rc;
  if ((rc = make_mhd(m, vf, sf, powell, "dg_mesh_create_mhd_curved: cudaMalloc")) != DG_OK)
    return rc;
  *out = m;
  return DG_OK;
}

int dg_set_source(dg_mesh* m, int kind) {
  if (!valid_mesh(m)) return fail(DG_ERR_ARG, "dg_set_source: invalid mesh");
  if (kind != DG_SOURCE_NONE && kind != DG_SOURCE_MANUFACTURED)
    return fail(DG_ERR_ARG, "dg_set_source: unknown source %d", kind);
  if (kind != DG_SOURCE_NONE && (!m->curved || m->mhd))
    return fail(DG_ERR_ARG, "dg_set_source: source terms need a mesh from dg_mesh_create_curved");
  m->source = kind;
  if (m->graph) {  // a recorded step holds the old source choice
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  return DG_OK;
}

int dg_set_time(dg_mesh* m, double t) {
  if (!valid_mesh(m) || !isfinite(t)) return fail(DG_ERR_ARG, "dg_set_time: bad argument");
  set_dt_kernel<<<1, 1, 0, m->stream>>>(m->t_dev, t);
  DG_CUDA(cudaGetLastError(), "dg_set_time: launch");
  return DG_OK;
}

int dg_get_time(dg_mesh* m, double* t) {
  if (!valid_mesh(m) || !t) return fail(DG_ERR_ARG, "dg_get_time: bad argument");
  DG_CUDA(cudaMemcpyAsync(t, m->t_dev, sizeof(double), cudaMemcpyDeviceToHost, m->stream),
          "dg_get_time: copy");
  DG_CUDA(cudaStreamSynchronize(m->stream), "dg_get_time: sync");
  return DG_OK;
}

int dg_mesh_destroy(dg_mesh* m) {
  if (!m) return DG_OK;
  cudaStreamSynchronize(m->stream);
  cudaFree(m->k);
  cudaFree(m->fs);
  cudaFree(m->wq);
  cudaFree(m->partials);
  cudaFree(m->red_out);
  cudaFree(m->speed);
  cudaFree(m->err);
  cudaFree(m->fbar);
  cudaFree(m->ref);
  cudaFree(m->refE);
  cudaFree(m->dt_dev);
  cudaFree(m->u_dev);
  cudaFree(m->t_dev);
  cudaFree(m->pp_buf);
  cudaFree(m->Ja);
  cudaFree(m->invJ);
  cudaFree(m->Jdet);
  cudaFree(m->X);
  if (m->graph) cudaGraphExecDestroy(m->graph);
  delete m;
  return DG_OK;
}

int dg_mesh_info(const dg_mesh* m, long long* n_nodes, int* n_vars, long long* n_values) {
  if (!valid_mesh(m)) return fail(DG_ERR_ARG, "dg_mesh_info: invalid mesh");
  if (n_nodes) *n_nodes = m->nnodes;
  if (n_vars) *n_vars = m->nv;
  if (n_values) *n_values = m->nvalues;
  return DG_OK;
}

int dg_mesh_set_stream(dg_mesh* m, void* cuda_stream) {
  if (!valid_mesh(m)) return fail(DG_ERR_ARG, "dg_mesh_set_stream: invalid mesh");
  m->stream = (cudaStream_t)cuda_stream;
  return DG_OK;
}

int dg_rhs(dg_mesh* m, const double* u, void* du) { return dg_rhs_part(m, u, du, 3); }

int dg_rhs_part(dg_mesh* m, const double* u, void* du, int parts) {
  if (!valid_mesh(m) || !u || !du) return fail(DG_ERR_ARG, "dg_rhs: null argument");
  if (parts < 1 || (parts > 3 && parts != 6))
    return fail(DG_ERR_ARG, "dg_rhs_part: parts must be 1, 2, 3 or 6");
  dg::StageFuse fz;
  if (parts == 6) {
    // the volume kernel with the stage update fused in, as in stages 2-5
    // (A != 0 reads k): k <- k + dt du, u unchanged (times the kernel of the
    // fused step)
    fz.k = m->k;
    fz.dt = m->dt_dev;
    fz.a = 1.0;
    fz.b = 0.0;
    parts = 2;
  }
  cudaError_t e;
  if (m->mhd && m->curved) {
    e = dg::mhd_curved_rhs_launch(m->N, u, (double*)du, (double*)m->fs, m->Ja, m->invJ, m->geom,
                                  m->ctab, m->mhd_vf, m->powell, m->mhd_sf, m->err, m->stream,
                                  parts, fz);
  } else if (m->mhd) {
    e = dg::mhd_rhs_launch(m->N, u, (double*)du, (double*)m->fs, m->geom, m->tmhd, m->t64, m->mhd_vf, m->powell, m->mhd_sf,
                           m->err, m->stream, parts, fz);
  } else if (m->curved) {
    dg::SourceArgs src;  // the source at the mesh time
    src.kind = m->source;
    src.t0 = m->t_dev;
    e = dg::curved_rhs_launch(m->N, const_cast<double*>(u), (double*)du, (double*)m->fs, m->Ja,
                              m->invJ, m->X, m->geom, m->ctab, m->opt.volume_flux,
                              m->opt.surface_flux, m->err, m->stream, parts, fz, src);
  } else if (m->opt.precision == DG_FP64) {
    e = (m->d == 2 ? dg::rhs_launch_double_2 : dg::rhs_launch_double_3)(
        m->N, u, (double*)du, (double*)m->fs, m->geom, m->t64, m->opt.volume_flux,
        m->opt.surface_flux, m->err, m->stream, parts, fz);
  } else {
    fz.ref = m->ref;
    fz.refE = m->refE;
    e = (m->d == 2 ? dg::rhs_launch_float_2 : dg::rhs_launch_float_3)(
        m->N, u, (float*)du, (float*)m->fs, m->geom, m->t32, m->opt.volume_flux,
        m->opt.surface_flux, m->err, m->stream, parts, fz);
  }
  if (e != cudaSuccess) return cuda_fail(e, "dg_rhs: launch");
  return DG_OK;
}

int dg_rhs_vjp(dg_mesh* m, const double* u, const double* w, double* ubar) {
  if (!valid_mesh(m) || !u || !w || !ubar) return fail(DG_ERR_ARG, "dg_rhs_vjp: null argument");
  if (m->curved || m->mhd)
    return fail(DG_ERR_ARG, "dg_rhs_vjp: not available on curved or MHD meshes");
  if (!m->fbar) {
    const long long n = 2LL * m->d * m->nv * m->nelem * (m->P / m->np);
    DG_CUDA(cudaMalloc(&m->fbar, n * sizeof(double)), "dg_rhs_vjp: cudaMalloc");
  }
  cudaError_t e;
  if (m->opt.precision == DG_FP64)
    e = (m->d == 2 ? dg::vjp_launch_double_2 : dg::vjp_launch_double_3)(
        m->N, u, w, ubar, m->fbar, m->geom, m->t64, m->opt.volume_flux, m->opt.surface_flux,
        m->stream);
  else
    e = (m->d == 2 ? dg::vjp_launch_float_2 : dg::vjp_launch_float_3)(
        m->N, u, w, ubar, m->fbar, m->geom, m->t64, m->opt.volume_flux, m->opt.surface_flux,
        m->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_rhs_vjp: launch");
  return DG_OK;
}

int dg_rk_stage(dg_mesh* m, double* u, const void* du, double a, double b, double dt) {
  if (!valid_mesh(m) || !u || !du) return fail(DG_ERR_ARG, "dg_rk_stage: null argument");
  const int grid = grid_for((m->nvalues + 1) / 2, 256);
  if (m->opt.precision == DG_FP64)
    rk_stage_kernel<double><<<grid, 256, 0, m->stream>>>(u, m->k, (const double*)du, a, b, dt,
                                                         m->nvalues);
  else
    rk_stage_kernel<float><<<grid, 256, 0, m->stream>>>(u, m->k, (const float*)du, a, b, dt,
                                                        m->nvalues);
  DG_CUDA(cudaGetLastError(), "dg_rk_stage: launch");
  return DG_OK;
}

int dg_rk_reset(dg_mesh* m) {
  if (!valid_mesh(m)) return fail(DG_ERR_ARG, "dg_rk_reset: invalid mesh");
  DG_CUDA(cudaMemsetAsync(m->k, 0, m->nvalues * sizeof(double), m->stream), "dg_rk_reset");
  return DG_OK;
}

int dg_step(dg_mesh* m, double* u, void* du, double dt) {
  if (!valid_mesh(m) || !u || !du) return fail(DG_ERR_ARG, "dg_step: null argument");
  if (m->curved && !m->mhd) {
    // source terms at the stage times t + c_s dt; the mesh time advances by dt
    set_dt_kernel<<<1, 1, 0, m->stream>>>(m->dt_dev, dt);
    DG_CUDA(cudaGetLastError(), "dg_step: launch");
    for (int s = 0; s < 5; ++s) {
      dg::SourceArgs src;
      src.kind = m->source;
      src.t0 = m->t_dev;
      src.dt = m->dt_dev;
      src.c = kRkC[s];
      DG_CUDA(dg::curved_rhs_launch(m->N, u, (double*)du, (double*)m->fs, m->Ja, m->invJ, m->X,
                                    m->geom, m->ctab, m->opt.volume_flux, m->opt.surface_flux,
                                    m->err, m->stream, 3, dg::StageFuse(), src),
              "dg_step: rhs launch");
      const int rc = dg_rk_stage(m, u, du, kRkA[s], kRkB[s], dt);
      if (rc != DG_OK) return rc;
    }
    advance_time_kernel<<<1, 1, 0, m->stream>>>(m->t_dev, m->dt_dev);
    DG_CUDA(cudaGetLastError(), "dg_step: launch");
    return DG_OK;
  }
  for (int s = 0; s < 5; ++s) {
    int rc = dg_rhs(m, u, du);
    if (rc != DG_OK) return rc;
    rc = dg_rk_stage(m, u, du, kRkA[s], kRkB[s], dt);
    if (rc != DG_OK) return rc;
  }
  return DG_OK;
}

namespace {

// dt on the device, then five stages with the update fused into the volume
// kernel (no du buffer, no host synchronisation)

// The five fused stages on the device state u with the time step in
// m->dt_dev; out (optional): where the last stage stores the new state.
int enqueue_fused_stages(dg_mesh* m, double* u, double* out) {
  // small FP64 Cartesian meshes run each stage as one launch (faces and
  // volume) from one buffer into another: u -> A -> B -> A -> B -> u (or out)
  const bool pp = m->pp_buf && !m->mhd && !m->curved && m->opt.precision == DG_FP64;
  double* const A = pp ? m->pp_buf : nullptr;
  double* const B = pp ? m->pp_buf + m->nvalues : nullptr;
  for (int s = 0; s < 5; ++s) {
    dg::StageFuse fz;
    fz.k = m->k;
    fz.dt = m->dt_dev;
    fz.a = kRkA[s];
    fz.b = kRkB[s];
    if (s == 4) fz.u_out = out;
    double* const u_in = !pp ? u : (s == 0 ? u : (s % 2 == 1 ? A : B));
    if (pp) fz.u_out = s == 4 ? (out ? out : u) : (s % 2 == 0 ? A : B);
    cudaError_t e;
    if (m->mhd && m->curved) {
      e = dg::mhd_curved_rhs_launch(m->N, u, nullptr, (double*)m->fs, m->Ja, m->invJ, m->geom,
                                    m->ctab, m->mhd_vf, m->powell, m->mhd_sf, m->err, m->stream,
                                    3, fz);
    } else if (m->mhd) {
      e = dg::mhd_rhs_launch(m->N, u, nullptr, (double*)m->fs, m->geom, m->tmhd, m->t64, m->mhd_vf, m->powell, m->mhd_sf,
                             m->err, m->stream, 3, fz);
    } else if (m->curved) {
      dg::SourceArgs src;  // stage time t + c_s dt
      src.kind = m->source;
      src.t0 = m->t_dev;
      src.dt = m->dt_dev;
      src.c = kRkC[s];
      e = dg::curved_rhs_launch(m->N, u, nullptr, (double*)m->fs, m->Ja, m->invJ, m->X, m->geom,
                                m->ctab, m->opt.volume_flux, m->opt.surface_flux, m->err,
                                m->stream, 3, fz, src);
    } else if (m->opt.precision == DG_FP64) {
      e = (m->d == 2 ? dg::rhs_launch_double_2 : dg::rhs_launch_double_3)(
          m->N, u_in, nullptr, (double*)m->fs, m->geom, m->t64, m->opt.volume_flux,
          m->opt.surface_flux, m->err, m->stream, 3, fz);
    } else {
      fz.ref = m->ref;
      fz.refE = m->refE;
      e = (m->d == 2 ? dg::rhs_launch_float_2 : dg::rhs_launch_float_3)(
          m->N, u, nullptr, (float*)m->fs, m->geom, m->t32, m->opt.volume_flux,
          m->opt.surface_flux, m->err, m->stream, 3, fz);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fused stage launch");
  }
  if (m->curved) {
    advance_time_kernel<<<1, 1, 0, m->stream>>>(m->t_dev, m->dt_dev);
    DG_CUDA(cudaGetLastError(), "time advance launch");
  }
  return DG_OK;
}

// One CFL step on the device state u. src (optional): where the step's
// input state is read by the wave-speed pass, which then copies it into u;
// out (optional): where the last stage stores the new state instead of u.
int enqueue_fused_step(dg_mesh* m, double* u, double cfl, const double* src = nullptr,
                       double* out = nullptr) {
  bool dt_done = false;
  int rc = src ? launch_speed(m, src, u, cfl, &dt_done) : launch_speed(m, u, nullptr, cfl, &dt_done);
  if (rc) return rc;
  if (!dt_done) {
    dt_kernel<<<1, 1, 0, m->stream>>>(m->speed, m->N, cfl, m->dt_dev, m->err);
    DG_CUDA(cudaGetLastError(), "dt kernel launch");
  }
  return enqueue_fused_stages(m, u, out);
}
}  // namespace

int dg_step_dt(dg_mesh* m, double* u, double dt) {
  if (!valid_mesh(m) || !u || !(dt > 0.0)) return fail(DG_ERR_ARG, "dg_step_dt: bad argument");
  set_dt_kernel<<<1, 1, 0, m->stream>>>(m->dt_dev, dt);
  DG_CUDA(cudaGetLastError(), "dg_step_dt: launch");
  return enqueue_fused_stages(m, u, nullptr);
}

int dg_step_cfl(dg_mesh* m, double* u, double cfl) {
  if (!valid_mesh(m) || !u || !(cfl > 0.0)) return fail(DG_ERR_ARG, "dg_step_cfl: bad argument");
  return enqueue_fused_step(m, u, cfl);
}

int dg_step_graph(dg_mesh* m, double* u, double cfl) {
  if (!valid_mesh(m) || !u || !(cfl > 0.0)) return fail(DG_ERR_ARG, "dg_step_graph: bad argument");
  if (!m->graph || m->graph_u != u || m->graph_cfl != cfl) {
    if (m->graph) {
      cudaGraphExecDestroy(m->graph);
      m->graph = nullptr;
    }
    cudaStream_t cap;
    DG_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "dg_step_graph: stream");
    cudaStream_t saved = m->stream;
    m->stream = cap;
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = (ce == cudaSuccess) ? enqueue_fused_step(m, u, cfl) : DG_ERR_CUDA;
    if (ce == cudaSuccess) ce = cudaStreamEndCapture(cap, &g);
    m->stream = saved;
    cudaStreamDestroy(cap);
    if (rc != DG_OK || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != DG_OK ? rc : cuda_fail(ce, "dg_step_graph: capture");
    }
    ce = cudaGraphInstantiate(&m->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "dg_step_graph: instantiate");
    m->graph_u = u;
    m->graph_cfl = cfl;
  }
  DG_CUDA(cudaGraphLaunch(m->graph, m->stream), "dg_step_graph: launch");
  return DG_OK;
}

int dg_step_cfl_host(dg_mesh* m, double* u_host, double cfl, int n_steps) {
  if (!valid_mesh(m) || !u_host || !(cfl > 0.0) || n_steps < 1)
    return fail(DG_ERR_ARG, "dg_step_cfl_host: bad argument");
  cudaPointerAttributes pa;
  DG_CUDA(cudaPointerGetAttributes(&pa, u_host), "dg_step_cfl_host: pointer attributes");
  if (pa.type == cudaMemoryTypeDevice)
    return fail(DG_ERR_ARG, "dg_step_cfl_host: u_host is device memory (use dg_step_cfl)");
  if (!m->u_dev)
    DG_CUDA(cudaMalloc(&m->u_dev, sizeof(double) * m->nvalues), "dg_step_cfl_host: alloc");
  const size_t bytes = sizeof(double) * m->nvalues;
  // pinned and mapped: the first wave-speed pass reads the host buffer and
  // fills the device copy, the last stage stores the new state into it
  const bool mapped = pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr;
  double* hdev = mapped ? static_cast<double*>(pa.devicePointer) : nullptr;
  if (!mapped)
    DG_CUDA(cudaMemcpyAsync(m->u_dev, u_host, bytes, cudaMemcpyHostToDevice, m->stream),
            "dg_step_cfl_host: copy in");
  for (int i = 0; i < n_steps; ++i) {
    const double* src = (mapped && i == 0) ? hdev : nullptr;
    double* out = (mapped && i == n_steps - 1) ? hdev : nullptr;
    const int rc = enqueue_fused_step(m, m->u_dev, cfl, src, out);
    if (rc) return rc;
  }
  if (!mapped)
    DG_CUDA(cudaMemcpyAsync(u_host, m->u_dev, bytes, cudaMemcpyDeviceToHost, m->stream),
            "dg_step_cfl_host: copy out");
  DG_CUDA(cudaStreamSynchronize(m->stream), "dg_step_cfl_host: sync");
  return DG_OK;
}

int dg_last_dt(dg_mesh* m, double* dt_out) {
  if (!valid_mesh(m) || !dt_out) return fail(DG_ERR_ARG, "dg_last_dt: bad argument");
  DG_CUDA(cudaMemcpyAsync(dt_out, m->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, m->stream),
          "dg_last_dt: copy");
  DG_CUDA(cudaStreamSynchronize(m->stream), "dg_last_dt: sync");
  return DG_OK;
}

int dg_mesh_check(dg_mesh* m, int* flags) {
  if (!valid_mesh(m)) return fail(DG_ERR_ARG, "dg_mesh_check: invalid mesh");
  unsigned h = 0;
  DG_CUDA(cudaMemcpyAsync(&h, m->err, sizeof(unsigned), cudaMemcpyDeviceToHost, m->stream),
          "dg_mesh_check: copy");
  DG_CUDA(cudaStreamSynchronize(m->stream), "dg_mesh_check: sync");
  if (flags) *flags = (int)h;
  if (h) {
    DG_CUDA(cudaMemsetAsync(m->err, 0, sizeof(unsigned), m->stream), "dg_mesh_check: clear");
    return fail(DG_ERR_NONPHYSICAL, "non-physical state met (flags %u: 1 rho<=0, 2 p<=0, 4 NaN)", h);
  }
  return DG_OK;
}

int dg_max_dt(dg_mesh* m, const double* u, double cfl, double* dt_out) {
  if (!valid_mesh(m) || !u || !dt_out || !(cfl > 0.0))
    return fail(DG_ERR_ARG, "dg_max_dt: bad argument");
  DG_CUDA(cudaMemsetAsync(m->speed, 0, sizeof(unsigned long long), m->stream), "dg_max_dt: clear");
  int rc0 = launch_speed(m, u);
  if (rc0) return rc0;
  unsigned long long bits = 0;
  DG_CUDA(cudaMemcpyAsync(&bits, m->speed, sizeof(bits), cudaMemcpyDeviceToHost, m->stream),
          "dg_max_dt: copy");
  int rc = dg_mesh_check(m, nullptr);
  if (rc != DG_OK) return rc;
  double worst;
  memcpy(&worst, &bits, sizeof(worst));
  if (!(worst > 0.0)) return fail(DG_ERR_NONPHYSICAL, "dg_max_dt: zero or invalid wave speed");
  *dt_out = cfl * 2.0 / ((m->N + 1) * worst);
  return DG_OK;
}

int dg_integrals(dg_mesh* m, const double* u, double* out) {
  if (!valid_mesh(m) || !u || !out) return fail(DG_ERR_ARG, "dg_integrals: null argument");
  if (m->mhd) return fail(DG_ERR_ARG, "dg_integrals: not available on MHD meshes");
  const int nq = m->d + 4;
  if (m->d == 2)
    integrals_kernel<2><<<kRedBlocks, kRedThreads, 0, m->stream>>>(u, m->geom, (int)m->P, m->wq,
                                                                   m->Jdet, m->partials, m->err);
  else
    integrals_kernel<3><<<kRedBlocks, kRedThreads, 0, m->stream>>>(u, m->geom, (int)m->P, m->wq,
                                                                   m->Jdet, m->partials, m->err);
  DG_CUDA(cudaGetLastError(), "dg_integrals: launch");
  integrals_final_kernel<<<1, kRedThreads, 0, m->stream>>>(m->partials, kRedBlocks, nq,
                                                           m->red_out);
  DG_CUDA(cudaGetLastError(), "dg_integrals: final launch");
  double host[14];
  DG_CUDA(cudaMemcpyAsync(host, m->red_out, 2 * nq * sizeof(double), cudaMemcpyDeviceToHost,
                          m->stream),
          "dg_integrals: copy");
  int rc = dg_mesh_check(m, nullptr);
  if (rc != DG_OK) return rc;
  for (int q = 0; q < nq; ++q) out[q] = host[2 * q] + host[2 * q + 1];
  return DG_OK;
}

}  // extern "C"
