// dg_rhs_noalloc: the FP64 rhs for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code embedded in another
// runtime that owns every device allocation through its own arena, plugins
// that run under a memory budget fixed at load time, or callers that must
// not allocate once their setup phase is over. dg_mesh_create allocates the
// face-flux scratch and other buffers, so this entry point takes the mesh as
// plain arguments and keeps its scratch -- the surface-flux buffer and the
// device error word -- in one file-scope static device array
// (kStaticValues doubles, 16 MiB). The array is claimed in a CUDA context
// when this file's module is loaded there (with lazy module loading, at the
// first call in that context) and is held until the context ends.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include "dgsem.h"
#include "dg_device.cuh"

namespace dg {
cudaError_t rhs_launch_double_2(int, const double*, double*, double*, const Geom&,
                                const Tables<double>&, int, int, unsigned*, cudaStream_t, int,
                                const StageFuse&);
cudaError_t rhs_launch_double_3(int, const double*, double*, double*, const Geom&,
                                const Tables<double>&, int, int, unsigned*, cudaStream_t, int,
                                const StageFuse&);
int set_last_error(int code, const char* msg);
void build_tables_fp64(int d, int N, const double* h, Tables<double>* t);
}  // namespace dg

namespace {

// face values d (d+2) n_elem (N+1)^(d-1) must fit in kFaceValues; one more
// slot (the last double) holds the device error word
constexpr long long kFaceValues = (1LL << 21) - 32;
constexpr long long kStaticValues = 1LL << 21;  // 16 MiB of doubles

static __device__ __align__(256) double g_noalloc_scratch[kStaticValues];

int fail(int code, const char* fmt, long long a = 0, long long b = 0) {
  char buf[256];
  snprintf(buf, sizeof(buf), fmt, a, b);
  return dg::set_last_error(code, buf);
}

// Device address of the static scratch in the current context. In host code
// the array's name is only a host-side stand-in, so the address is looked up
// on every call: nothing is cached that could outlive a context (after
// cudaDeviceReset, or under a caller's own non-primary context). Once the
// module is loaded in the context the lookup allocates nothing; the first
// lookup loads it and claims the array, and fails if the device has no room.
int scratch_in_current_context(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e == cudaErrorMemoryAllocation)
    return fail(DG_ERR_CUDA,
                "dg_rhs_noalloc: the device has no room for the 16 MiB static scratch "
                "(claimed when the module loads, at the first call in a context)");
  if (e != cudaSuccess || !p)
    return fail(DG_ERR_CUDA, "dg_rhs_noalloc: cudaGetSymbolAddress failed (error %lld)",
                (long long)e);
  *out = static_cast<double*>(p);
  return DG_OK;
}

}  // namespace

extern "C" int dg_rhs_noalloc(int d, int N, const int* elements_per_dim, const double* domain,
                              const dg_options* opt, const double* u, double* du,
                              void* cuda_stream) {
  if (!elements_per_dim || !domain || !u || !du)
    return fail(DG_ERR_ARG, "dg_rhs_noalloc: null argument");
  if (d < 2 || d > 3) return fail(DG_ERR_ARG, "dg_rhs_noalloc: d must be 2 or 3 (got %lld)", d);
  if (N < 1 || N > 7) return fail(DG_ERR_ARG, "dg_rhs_noalloc: N must be in [1, 7] (got %lld)", N);
  dg_options o = {1.4, DG_VFLUX_RANOCHA, DG_SFLUX_LLF, DG_FP64};
  if (opt) o = *opt;
  if (!(o.gamma > 1.0) || o.volume_flux < 0 || o.volume_flux > 2 || o.surface_flux < 0 ||
      o.surface_flux > 3 || o.precision != DG_FP64)
    return fail(DG_ERR_ARG, "dg_rhs_noalloc: invalid options (only DG_FP64 precision)");
  dg::Geom g;
  double h[3] = {1.0, 1.0, 1.0};
  g.n[0] = g.n[1] = g.n[2] = 1;
  g.nelem = 1;
  long long lines = 1;
  for (int k = 0; k < d; ++k) {
    if (elements_per_dim[k] < 1 || !(domain[2 * k + 1] > domain[2 * k]))
      return fail(DG_ERR_ARG, "dg_rhs_noalloc: bad elements_per_dim or domain in direction %lld", k);
    g.n[k] = elements_per_dim[k];
    g.nelem *= elements_per_dim[k];
    h[k] = (domain[2 * k + 1] - domain[2 * k]) / elements_per_dim[k];
    if (k > 0) lines *= (N + 1);
    if (g.nelem > kFaceValues) break;
  }
  g.gamma = o.gamma;
  g.gm1 = o.gamma - 1.0;
  g.gm1inv = 1.0 / (o.gamma - 1.0);
  const long long face_values = (long long)d * (d + 2) * g.nelem * lines;
  if (g.nelem > kFaceValues || face_values > kFaceValues)
    return fail(DG_ERR_ARG,
                "dg_rhs_noalloc: mesh needs %lld face values, more than the static scratch "
                "holds (%lld); use dg_mesh_create/dg_rhs for larger meshes",
                face_values, kFaceValues);
  double* scratch = nullptr;
  int rc = scratch_in_current_context(&scratch);
  if (rc != DG_OK) return rc;
  unsigned* err = reinterpret_cast<unsigned*>(scratch + kFaceValues);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the error word must start at zero; the face buffer is fully rewritten by
  // the surface kernel before the volume kernel reads it
  if (cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess)
    return fail(DG_ERR_CUDA, "dg_rhs_noalloc: clearing the error word failed");
  dg::Tables<double> tb;
  dg::build_tables_fp64(d, N, h, &tb);
  cudaError_t e = (d == 2 ? dg::rhs_launch_double_2 : dg::rhs_launch_double_3)(
      N, u, du, scratch, g, tb, o.volume_flux, o.surface_flux, err, st, 3, dg::StageFuse());
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, "dg_rhs_noalloc: launch failed");
  return DG_OK;
}
