/*
 * dgsem.h - C ABI of the GB300 (sm_103a) DGSEM library: the right-hand side
 * du/dt = rhs(u) of the discontinuous Galerkin spectral element method for the
 * 2D/3D compressible Euler equations (ideal gas) on a uniform periodic
 * Cartesian mesh or on the warped periodic box of the paper's benchmark (3D),
 * the same for the 3D ideal MHD equations, and the low-storage Runge-Kutta
 * stage that consumes it.
 *
 * Paper: H. Ranocha et al., "Adaptive numerical simulations with Trixi.jl: A
 * case study of Julia for scientific computing" (2021).
 *   - conservation law d_t u + sum_j d_xj f^j(u) = 0: Sec. 2, Eq. (1);
 *   - DGSEM on LGL nodes, entropy-conservative flux differencing with the
 *     Ranocha EC/KEP two-point flux: Sec. 2.1 and Sec. 3.1;
 *   - surface fluxes (local Lax-Friedrichs, EC, HLL): Sec. 2.2, Sec. 3.1;
 *   - Carpenter-Kennedy 5-stage 4th-order low-storage RK and the CFL time
 *     step: Sec. 3.1; performance index PID: Sec. 3.1, Eq. (3);
 *   - the curvilinear benchmark mesh (warped periodic box) and its
 *     manufactured-solution problem: Sec. 3.1;
 *   - analysis integrals: Sec. 2.2;
 *   - 3D ideal MHD for the Alfven-wave runs, the weak form and EC flux
 *     differencing with the Powell non-conservative term, HLL/LLF/EC faces,
 *     on the Cartesian mesh and the warped box: Sec. 3.1.
 *
 * Conventions shared by every entry point:
 *   - State layout u[e][v][k][j][i]: element-major; inside an element the
 *     d+2 conserved variables (rho, rho v_1..rho v_d, E) one after another
 *     (eight, (rho, rho v, E, B), on an MHD mesh),
 *     each as (N+1)^d nodal values with i (x) fastest. Elements are ordered
 *     lexicographically with x fastest: e = ex + n0 (ey + n1 ez). Element
 *     (ex, ey, ez) covers [lo + ex h, lo + (ex+1) h] in each direction.
 *   - Buffers passed to compute calls are DEVICE pointers owned by the caller
 *     (the library never frees them), at least 16-byte aligned; the one
 *     exception, dg_step_cfl_host, takes a host buffer. The state u
 *     is always float64. The rhs output du is float64 in DG_FP64 precision and
 *     float32 in DG_FP32 precision.
 *   - The library owns the mesh object and its device scratch: the RK
 *     register k, the surface-flux buffer, the reduction partials and a
 *     device error word.
 *   - Compute calls are asynchronous on the mesh's CUDA stream unless they
 *     return host values (dg_max_dt, dg_integrals, dg_mesh_check), which
 *     synchronise that stream.
 *   - Every call returns a dg_status; nothing is thrown or aborted across the
 *     ABI. dg_last_error() gives a thread-local message for the last failure.
 */
#ifndef DGSEM_H
#define DGSEM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh dg_mesh; /* opaque, library-owned */

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,         /* invalid argument: handle, size, pointer, option */
  DG_ERR_CUDA = -2,        /* a CUDA runtime call failed */
  DG_ERR_OOM = -3,         /* device allocation failed */
  DG_ERR_NONPHYSICAL = -4, /* rho <= 0, p <= 0 or a non-finite value was met */
  DG_ERR_TIMEOUT = -5      /* a bounded device wait gave up */
} dg_status;

/* Two-point volume fluxes (flux differencing, Sec. 2.1/3.1). DG_VFLUX_EC is
 * the entropy-conservative MHD flux (MHD meshes only). */
enum { DG_VFLUX_RANOCHA = 0, DG_VFLUX_CHANDRASHEKAR = 1, DG_VFLUX_CENTRAL = 2, DG_VFLUX_EC = 3 };
/* Surface fluxes. LLF wave speed: max(|v_n,L|, |v_n,R|) + max(c_L, c_R).
 * DG_SFLUX_EC is the entropy-conservative MHD flux (MHD meshes only). */
enum {
  DG_SFLUX_LLF = 0,
  DG_SFLUX_RANOCHA = 1,
  DG_SFLUX_HLL = 2,
  DG_SFLUX_CHANDRASHEKAR = 3,
  DG_SFLUX_EC = 4
};
/* Arithmetic of the rhs kernels. RK accumulation and reductions are FP64. */
enum { DG_FP64 = 0, DG_FP32 = 1 };

typedef struct {
  double gamma;     /* ratio of specific heats, > 1 */
  int volume_flux;  /* DG_VFLUX_* */
  int surface_flux; /* DG_SFLUX_* */
  int precision;    /* DG_FP64 or DG_FP32 */
} dg_options;

/* Create a uniform periodic Cartesian mesh of elements_per_dim[0] x ... x
 * elements_per_dim[d-1] elements of polynomial degree N on the box
 * domain = {lo_0, hi_0, lo_1, hi_1[, lo_2, hi_2]}.
 * d in {2, 3}; 1 <= N <= 7; every elements_per_dim[k] >= 1; lo_k < hi_k.
 * opt NULL selects gamma = 1.4, Ranocha volume flux, LLF surface flux, FP64.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * Allocates the library-owned device buffers. Errors: DG_ERR_ARG, DG_ERR_OOM,
 * DG_ERR_CUDA; *out is NULL on failure. */
int dg_mesh_create(int d, int N, const int *elements_per_dim, const double *domain,
                   const dg_options *opt, void *cuda_stream, dg_mesh **out);

/* Create the curvilinear mesh of the paper's performance benchmark
 * (Sec. 3.1): the periodic box [-1,1]^3 of elements_per_dim[0] x [1] x [2]
 * elements of degree N (1..7) whose interior is warped by
 *   y = eta  + warp cos(1.5 pi xi) cos(0.5 pi eta) cos(0.5 pi zeta),
 *   x = xi   + warp cos(0.5 pi xi) cos(2 pi y)    cos(0.5 pi zeta),
 *   z = zeta + warp cos(0.5 pi x)  cos(pi y)      cos(0.5 pi zeta)
 * ((xi, eta, zeta) the Cartesian coordinates of the box; warp = 0.15 in the
 * paper, 0 gives the Cartesian mesh). Each element is the image of the
 * reference cube under the degree-N interpolant of the mapping at the LGL
 * nodes; the library computes the metric terms in the conservative curl form
 * (free-stream preserving) and the Jacobians on the device. dg_rhs,
 * dg_rhs_part, dg_step, dg_step_cfl, dg_step_dt, dg_step_graph,
 * dg_step_cfl_host, dg_max_dt and dg_integrals accept such meshes (the
 * split-form operator with contravariant two-point fluxes, surface fluxes
 * along the left element's metric vector, du scaled by 1/J; the CFL rule with
 * contravariant wave speeds); dg_rhs_vjp does not. FP64 only
 * (opt->precision must be DG_FP64); 2D is not offered. Errors: DG_ERR_ARG
 * (also for |warp| > 0.5), DG_ERR_OOM, DG_ERR_CUDA. */
int dg_mesh_create_curved(int N, const int *elements_per_dim, double warp, const dg_options *opt,
                          void *cuda_stream, dg_mesh **out);

/* Replace the node coordinates of a curved mesh (dg_mesh_create_curved or
 * dg_mesh_create_mhd_curved) by X, a device float64 array [n_elem][3][P]
 * (per element the x, y and z coordinates of its P = (N+1)^3 nodes, node i
 * fastest; 8-byte aligned; the caller keeps ownership), and rebuild the
 * metric terms and Jacobians from them on the device with the same
 * construction (nodal derivatives, conservative curl form). The elements
 * keep their places in the periodic box: X must describe a valid mesh of
 * the same connectivity (positive Jacobians; the periodic faces matching).
 * Used to run the operator on coordinates computed elsewhere, e.g. by
 * another code's mesh generator (Sec. 3.1 mesh). Asynchronous on the mesh's
 * stream. Errors: DG_ERR_ARG (not a curved mesh, null or misaligned X),
 * DG_ERR_CUDA. */
int dg_mesh_set_nodes(dg_mesh *mesh, const double *X);

/* Replace the metric terms and Jacobians of a curved mesh by the caller's:
 * Ja device float64 [n_elem][3][3][P] with Ja[e][r][n][node] = (J a^r)_n (the
 * contravariant metric vector of reference direction r, physical component
 * n) and J device float64 [n_elem][P]; the library keeps copies and forms
 * 1/J. For operators on geometry computed elsewhere (call after
 * dg_mesh_set_nodes, whose coordinates the source terms use). Asynchronous
 * on the mesh's stream. Errors: DG_ERR_ARG (not a curved mesh, null
 * pointer), DG_ERR_CUDA. */
int dg_mesh_set_metric(dg_mesh *mesh, const double *Ja, const double *J);

/* Create a uniform periodic Cartesian mesh (as dg_mesh_create with d = 3) for
 * the 3D ideal MHD equations, u = (rho, rho v_1..3, E, B_1..3), E = p/(gamma-1)
 * + rho |v|^2/2 + |B|^2/2 (the magnetic Alfven-wave setting of Sec. 3.1; the
 * paper gives no formulas, the discretisation below is this library's reading):
 *   - weak-form DGSEM: the split form with the central two-point flux
 *     (f(u_i) + f(u_m))/2, which is the strong-form derivative of the nodal
 *     flux; faces by local Lax-Friedrichs, lambda = max(|v_n,L|, |v_n,R|) +
 *     max(c_f,L, c_f,R), c_f the fast magnetosonic speed, or by HLL (the
 *     paper's weak-form coupling) with S_L = min(v_n,L - c_f,L, v_n,R -
 *     c_f,R), S_R = max(v_n,L + c_f,L, v_n,R + c_f,R);
 *   - powell = 1 adds the non-conservative term -(div B) (0, B, v.B, v), div B
 *     the same strong-form derivative of B_n with the interface average
 *     {B_n} at the faces; powell = 0 leaves the conservative system;
 *   - or flux differencing with the entropy-conservative two-point flux
 *     (opt->volume_flux = DG_VFLUX_EC; the paper's second MHD solver) that
 *     satisfies [[w]] . f + {B_n} [[theta]] = [[rho v_n + beta v_n |B|^2]]
 *     (w the entropy variables, theta = 2 beta v.B, beta = rho/(2p)), with
 *     the Powell term in the same split form; with DG_SFLUX_EC at the faces
 *     the semi-discrete entropy is conserved.
 * opt NULL selects gamma = 5/3, the weak form and LLF; otherwise
 * opt->volume_flux must be DG_VFLUX_CENTRAL or DG_VFLUX_EC, opt->surface_flux
 * DG_SFLUX_LLF, DG_SFLUX_HLL or DG_SFLUX_EC and opt->precision DG_FP64. 1 <= N <= 7. dg_rhs, dg_rhs_part, dg_rk_stage, dg_rk_reset,
 * dg_step, dg_step_dt, dg_step_cfl (CFL rule with |v_dir| + c_f,dir),
 * dg_step_graph, dg_step_cfl_host, dg_max_dt, dg_last_dt and dg_mesh_check
 * accept such meshes; dg_rhs_vjp, dg_integrals and dg_set_source do not
 * (DG_ERR_ARG). Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
int dg_mesh_create_mhd(int N, const int *elements_per_dim, const double *domain,
                       const dg_options *opt, int powell, void *cuda_stream, dg_mesh **out);

/* The MHD operators of dg_mesh_create_mhd on the warped periodic box of
 * dg_mesh_create_curved (the mesh of the paper's MHD performance runs,
 * Sec. 3.1; same warp rule, geometry computed on the device): two-point
 * fluxes along the mean metric vector of each node pair, sum_d g_d f#_d;
 * face fluxes along the metric vector of the left element's face node (LLF
 * and HLL in the unit direction scaled by its length, or EC); the Powell
 * divergence (1/J) times the split-form sums of g . (B_i + B_m)/2 and the
 * face terms {B} . g; du scaled by 1/J; the CFL rule with the contravariant
 * speeds |v . J a^r| + c_f |J a^r|. The same calls as on dg_mesh_create_mhd
 * meshes are accepted. Errors: DG_ERR_ARG (also for |warp| > 0.5),
 * DG_ERR_OOM, DG_ERR_CUDA. */
int dg_mesh_create_mhd_curved(int N, const int *elements_per_dim, double warp,
                              const dg_options *opt, int powell, void *cuda_stream,
                              dg_mesh **out);

/* Source terms (curved meshes only): DG_SOURCE_MANUFACTURED adds
 * S = d_t u + div F(u) of the manufactured solution rho = 2 + 0.1 sin(pi (x +
 * y + z - t)), v = (1, 1, 1), E = rho^2 (the smooth Euler problem of the
 * benchmark; the paper names it without a formula), evaluated at the node
 * coordinates and the mesh time: dg_rhs at the mesh time, the steps at the
 * stage times t + c_s dt. Errors: DG_ERR_ARG. */
enum { DG_SOURCE_NONE = 0, DG_SOURCE_MANUFACTURED = 1 };
int dg_set_source(dg_mesh *mesh, int kind);

/* Simulation time of the mesh (0 at creation; the steps of a curved mesh
 * advance it by their dt). dg_set_time is asynchronous, dg_get_time waits for
 * the mesh's stream. Errors: DG_ERR_ARG, DG_ERR_CUDA. */
int dg_set_time(dg_mesh *mesh, double t);
int dg_get_time(dg_mesh *mesh, double *t);

/* Free the mesh and its device buffers (after synchronising its stream).
 * NULL is accepted. */
int dg_mesh_destroy(dg_mesh *mesh);

/* Sizes: nodes M = n_elem (N+1)^d, variables V = d+2 (8 on an MHD mesh),
 * values V M. */
int dg_mesh_info(const dg_mesh *mesh, long long *n_nodes, int *n_vars, long long *n_values);

/* Change the CUDA stream used by subsequent calls on this mesh. */
int dg_mesh_set_stream(dg_mesh *mesh, void *cuda_stream);

/* The library's own LGL nodes xi[N+1] and weights w[N+1] (host arrays),
 * computed in long double and rounded (basis of Sec. 2.1's DGSEM). */
int dg_lgl_nodes(int N, double *xi, double *w);

/* du = rhs(u) (Sec. 2.1 DGSEM, Eq. (1) with s = 0): split-form flux
 * differencing in the volume, surface flux at every interface, lifting and
 * inverse-Jacobian scaling. u: device float64[n_values]; du: device
 * float64 (DG_FP64) or float32 (DG_FP32) [n_values]. Asynchronous.
 * Non-physical states set the device error word (see dg_mesh_check). */
int dg_rhs(dg_mesh *mesh, const double *u, void *du);

/* One kernel of dg_rhs, for timing the kernels separately: parts = 1
 * launches only the surface-flux kernel (fills the library's face buffer),
 * parts = 2 only the volume kernel with lifting (reads the face buffer of the
 * previous part-1 call on the same u), parts = 3 both (same as dg_rhs),
 * parts = 6 the volume kernel of the fused step (stage update in its
 * epilogue) as in stages 2-5, with coefficients A = 1, B = 0:
 * k <- k + dt du with the last device time step, u unchanged (read and
 * written back), du not written. Asynchronous. */
int dg_rhs_part(dg_mesh *mesh, const double *u, void *du, int parts);

/* Vector-Jacobian product of the rhs: ubar = (d rhs/d u)(u)^T w, for
 * differentiating through simulations (Sec. 2 feature list: automatic
 * differentiation of the semidiscretisation). u, w, ubar: device float64
 * [n_values], same layout as u. The two-point and surface-flux Jacobians are
 * recomputed with forward-mode dual numbers (nothing is kept from dg_rhs);
 * at non-smooth points max/min take the first argument on ties and
 * d|x|/dx = sign(x), sign(0) = +1. DG_FP32 meshes evaluate the Jacobians in
 * float. Allocates the face adjoint buffer on first use. Asynchronous. */
int dg_rhs_vjp(dg_mesh *mesh, const double *u, const double *w, double *ubar);

/* One stage of the Carpenter-Kennedy 2N-storage scheme (Sec. 3.1):
 * k <- a k + dt du; u <- u + b k, with the library-owned register k
 * (zeroed at creation and by dg_rk_reset). du has the rhs dtype of the mesh.
 * Asynchronous. */
int dg_rk_stage(dg_mesh *mesh, double *u, const void *du, double a, double b, double dt);

/* Zero the RK register k (start of a new integration). Asynchronous. */
int dg_rk_reset(dg_mesh *mesh);

/* One full LSRK step (5 stages of dg_rhs + dg_rk_stage with the published
 * Carpenter-Kennedy coefficients) using the caller's du buffer as scratch.
 * Asynchronous. */
int dg_step(dg_mesh *mesh, double *u, void *du, double dt);

/* One full LSRK step with the CFL time step computed on the device
 * (Sec. 3.1): a wave-speed reduction and the dt formula below run as kernels,
 * then five stages whose update k <- A k + dt du, u <- u + B k is fused into
 * the volume kernel (no du buffer, no host synchronisation). Asynchronous. */
int dg_step_cfl(dg_mesh *mesh, double *u, double cfl);

/* One full LSRK step with a given time step dt > 0 (Sec. 3.1 Carpenter-
 * Kennedy stages): the five stages of dg_step_cfl, the update fused into the
 * volume kernel, without the CFL reduction; dg_last_dt then returns dt.
 * Asynchronous. Errors: DG_ERR_ARG (null u, dt <= 0), DG_ERR_CUDA. */
int dg_step_dt(dg_mesh *mesh, double *u, double dt);

/* dg_step_cfl recorded once as a CUDA graph for (u, cfl) and replayed on
 * later calls with the same arguments. Asynchronous. */
int dg_step_graph(dg_mesh *mesh, double *u, double cfl);

/* n_steps >= 1 steps of dg_step_cfl on a state held in HOST memory: u_host
 * (n_values doubles, layout as dg_rhs) holds the state on entry and the
 * state after the steps on return. The library keeps a device copy
 * (n_values doubles, allocated on first use). When u_host is pinned and
 * mapped (cudaHostAlloc, or host memory registered with cudaHostRegister)
 * the first step's wave-speed pass reads it directly and fills the device
 * copy, and the last step's final stage stores the new state straight into
 * it, so the host-device traffic overlaps the kernels; other host memory is
 * copied in and out with cudaMemcpyAsync. Synchronous (returns once u_host
 * is written). A nonphysical state is reported by dg_mesh_check, as for
 * dg_step_cfl. Errors: DG_ERR_ARG (null pointer, cfl <= 0, n_steps < 1,
 * device memory), DG_ERR_OOM, DG_ERR_CUDA. */
int dg_step_cfl_host(dg_mesh *mesh, double *u_host, double cfl, int n_steps);

/* The time step used by the last dg_step_cfl / dg_step_graph (synchronises). */
int dg_last_dt(dg_mesh *mesh, double *dt_out);

/* CFL time step (Sec. 3.1): dt = cfl * 2 / ((N+1) max_e sum_k (2/h_k)
 * max_nodes(|v_k| + c)), c = sqrt(gamma p / rho). Synchronises the stream;
 * returns DG_ERR_NONPHYSICAL if the state is not physical. */
int dg_max_dt(dg_mesh *mesh, const double *u, double cfl, double *dt_out);

/* Integrals over the domain by each element's LGL quadrature (Sec. 2.2
 * analysis quantities): out[d+4] (host) = rho, rho v_1..rho v_d, E,
 * entropy S = -rho (ln p - gamma ln rho)/(gamma-1), kinetic energy
 * rho |v|^2 / 2. Compensated (double-double) reductions in FP64.
 * Synchronises the stream. */
int dg_integrals(dg_mesh *mesh, const double *u, double *out);

/* Synchronise the mesh's stream and report the device error word:
 * *flags (may be NULL) receives its bits (1 = rho <= 0, 2 = p <= 0,
 * 4 = non-finite); returns DG_ERR_NONPHYSICAL if any is set, and clears it. */
int dg_mesh_check(dg_mesh *mesh, int *flags);

/* dg_rhs without any device allocation, for callers that cannot allocate:
 * code running inside another runtime that owns all device memory through
 * its own arena, plugins with a memory budget fixed at load time, or callers
 * that may not allocate after their setup phase. (The paper has no
 * counterpart; it is an interface for such embedders.)
 * Same arithmetic as dg_rhs in DG_FP64 precision: the mesh is given as plain
 * arguments (as for dg_mesh_create; opt NULL = defaults, precision must be
 * DG_FP64) and u, du are caller-owned device float64 arrays of
 * (d+2) n_elem (N+1)^d values. The surface-flux scratch and the device error
 * word live in one static device array of 2^21 doubles (16 MiB). A CUDA
 * context claims it when the library's module for this entry point is loaded
 * there, which under lazy module loading is the first call in that context:
 * make that first call during setup (and before any stream capture). If the
 * device has no room for it then, that call returns DG_ERR_CUDA. The array is
 * held until the context ends (process exit or cudaDeviceReset). Meshes
 * needing more than 2^21 - 32 face values, d (d+2) n_elem (N+1)^(d-1), are
 * rejected with DG_ERR_ARG. No cudaMalloc, cudaFree or other allocating call
 * is made. The array's device address is looked up in the current context on
 * every call (no cached pointer, so a device reset or a caller-owned context
 * is safe). Every call shares the array and it keeps the last call's
 * contents: the error word is cleared at each call and non-physical states
 * are not reported by this entry point. Calls that overlap on the GPU (on
 * different streams, or from different threads) race on the shared scratch.
 * Asynchronous on cuda_stream. */
int dg_rhs_noalloc(int d, int N, const int *elements_per_dim, const double *domain,
                   const dg_options *opt, const double *u, double *du, void *cuda_stream);

/* ---- Batched ensemble of independent 3D periodic simulations ----
 * n_sims meshes of N[s] in {3,4,5} and elements_per_dim[s]^3 elements on the
 * boxes domains[6 s .. 6 s + 5] = {lo_0, hi_0, lo_1, hi_1, lo_2, hi_2}
 * (domains NULL: [-1,1]^3 for every member), the Sec. 3.1 setup (periodic
 * box, Carpenter-Kennedy LSRK, CFL step), advanced together. d[s] must be 3
 * (DG_ERR_ARG otherwise; d NULL means 3 for every member). The state of all
 * members is one float64 device array: member s occupies values
 * [offsets[s], offsets[s+1]) in the layout of u above.
 * Every Runge-Kutta stage is ONE cooperative kernel launch over a work list
 * of (member, element batch) items, in two phases separated by a grid-wide
 * barrier: the surface fluxes of all faces (each face once), then the
 * flux-differencing volume term, lifting and the stage update per element.
 * The barrier's wait is bounded (about one second): if it runs out the launch
 * stops and dg_ensemble_check returns DG_ERR_TIMEOUT. The arithmetic per
 * member is that of dg_rhs on the same mesh. Options: Ranocha volume flux
 * only; any surface flux; DG_FP64 or DG_FP32 arithmetic (FP64 state, FP32
 * in the perturbation form of dg_rhs). The library owns the RK register, the
 * face buffer and (FP32) the per-element reference states. */
typedef struct dg_ensemble dg_ensemble;

int dg_ensemble_create(int n_sims, const int *d, const int *N, const int *elements_per_dim,
                       const double *domains, const dg_options *opt, void *cuda_stream,
                       dg_ensemble **out);
int dg_ensemble_destroy(dg_ensemble *ens);
/* total values and nodes; offsets[n_sims+1] (may be NULL) */
int dg_ensemble_info(const dg_ensemble *ens, long long *n_values, long long *n_nodes,
                     long long *offsets);
/* per-member time steps: host arrays of n_sims (set / read back, synchronous) */
int dg_ensemble_set_dt(dg_ensemble *ens, const double *dt_host);
int dg_ensemble_get_dt(dg_ensemble *ens, double *dt_host);
/* per-member CFL time steps computed on the device from u (asynchronous;
 * the values stay on the device for the next stages) */
int dg_ensemble_compute_dt(dg_ensemble *ens, const double *u, double cfl);
/* one stage s in [0,5): u_out = u_in + B_s k, k = A_s k + dt du(u_in);
 * u_out may be u_in (in place). Asynchronous. */
int dg_ensemble_stage(dg_ensemble *ens, const double *u_in, double *u_out, int stage);
/* one full step in place on u (five in-place stages, no second buffer);
 * when cfl > 0 the time steps are first recomputed from u on the device. */
int dg_ensemble_step(dg_ensemble *ens, double *u, double cfl);
/* the same step recorded once as a CUDA graph (for this u and cfl) and
 * replayed on every later call. */
int dg_ensemble_step_graph(dg_ensemble *ens, double *u, double cfl);
int dg_ensemble_rk_reset(dg_ensemble *ens);
/* synchronise; DG_ERR_NONPHYSICAL if a non-physical state was met,
 * DG_ERR_TIMEOUT if a stage's barrier gave up; *flags gets the bits */
int dg_ensemble_check(dg_ensemble *ens, int *flags);
/* CTA shape: threads per CTA (multiple of 32, at most 128) and requested
 * resident CTAs per SM (the launch takes at most what fits); elements per
 * work item follow as threads / (N+1)^2 for each degree. */
int dg_ensemble_set_block(dg_ensemble *ens, int threads, int blocks_per_sm);
/* the current shape: threads per CTA, requested CTAs per SM, CTAs launched */
int dg_ensemble_get_block(const dg_ensemble *ens, int *threads, int *ctas_per_sm, int *grid);
/* threads per line of the volume phase (FP64 ensembles): on = 0, one thread
 * per element line walking its N(N+1)/2 node pairs (elements per work item
 * as above); on = 1, pair-parallel: the CTA takes the item's elements one
 * after another, one thread per (line, node pair) of a direction, then one
 * thread per node for the line sum (the same result, bitwise). DG_ERR_ARG
 * for on not in {0, 1} or on = 1 on an FP32 ensemble. */
int dg_ensemble_set_pair_parallel(dg_ensemble *ens, int on);
int dg_ensemble_get_pair_parallel(const dg_ensemble *ens, int *on);
/* autotuner: times one stage from u into u_tmp (u unchanged) for each
 * candidate (threads per CTA, CTAs per SM and, for FP64, the threads per
 * line above), keeps the fastest and reports it (outputs may be NULL; the
 * chosen threads per line: dg_ensemble_get_pair_parallel); k is preserved.
 * Allocates a copy of k for the trials. */
int dg_ensemble_tune(dg_ensemble *ens, const double *u, double *u_tmp, int *best_threads,
                     int *best_blocks_per_sm, float *best_ms);

/* Measurement helper for the roofline of the flux kernels (the paper has no
 * counterpart; its Sec. 3.1 performance index is a time per DOF): the FP64
 * and FP32 vector fused-multiply-add throughput of the current device in
 * TFLOP/s (an FMA counted as two flops), from a kernel of eight independent
 * FMA chains per thread, 8 CTAs of 256 threads per SM, timed with CUDA events
 * (the mean of three launches of at least 20 ms each), and the device's SM
 * count. Outputs may be NULL (that rate is then not measured). Synchronous
 * on cuda_stream; allocates nothing (the kernel's store target, never written
 * in practice, is a static device array of 4 MiB (FP64) and 2 MiB (FP32)).
 * Errors: DG_ERR_CUDA, DG_ERR_ARG (a device of more than 256 SMs). */
int dg_measure_peaks(double *fp64_tflops, double *fp32_tflops, int *sm_count, void *cuda_stream);

/* Measurement helper behind the layout of the small-mesh kernels (no paper
 * counterpart): the SM cycles per step of one dependent FP64 FMA chain run by
 * one warp per SM with all 32 lanes active (cycles_full_warp) and with one
 * lane active (cycles_one_lane), read with clock64 in the kernel. Equal
 * values mean that a warp's FP64 instruction costs the same whatever its
 * active lanes. Synchronous on cuda_stream; allocates nothing (a static
 * device array of two counters). Errors: DG_ERR_CUDA. Outputs may be NULL. */
int dg_measure_fp64_issue(double *cycles_full_warp, double *cycles_one_lane, void *cuda_stream);

/* Self-check of the library's device arithmetic helpers (no paper
 * counterpart; for the test suite): y[i] = f(x[i]) for n device doubles,
 * evaluated by the same device functions the kernels use:
 *   op 0  the FP64 reciprocal (hardware approximation + cubic Newton step),
 *   op 1  the FP32 reciprocal of (float)x[i], widened,
 *   op 2  the double -> float conversion of the FP32 kernels (integer pipe,
 *         round to nearest even), widened,
 *   op 3  the float -> double conversion of (float)x[i],
 *   op 4  the FP64 square root of the wave-speed kernels (hardware
 *         reciprocal-square-root approximation + Goldschmidt iteration).
 * Asynchronous on cuda_stream. Errors: DG_ERR_ARG, DG_ERR_CUDA. */
int dg_selftest_arith(int op, const double *x, double *y, long long n, void *cuda_stream);

/* Thread-local description of the last failed call ("" if none). */
const char *dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DGSEM_H */
