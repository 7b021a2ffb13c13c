// Launchers of the curvilinear-mesh kernels (dg_curved.cuh), degrees 1..7.
#include "dg_curved.cuh"

namespace dg {

namespace {

template <int N>
cudaError_t geometry_n(const CGeom& cg, double* Ja, double* invJ, double* Jdet, double* X,
                       cudaStream_t st) {
  constexpr int P = (N + 1) * (N + 1) * (N + 1);
  curved_geometry_kernel<N><<<(unsigned)cg.g.nelem, P, 0, st>>>(cg, Ja, invJ, Jdet, X);
  return cudaGetLastError();
}

template <int N, int VF, int EPB>
cudaError_t volume_epb(double* u, double* du, const double* fs, const double* Ja,
                       const double* invJ, const double* X, const Geom& g, const CTables& tb,
                       unsigned* err, cudaStream_t st, const StageFuse& fz,
                       const SourceArgs& src) {
  using L = CLaunch<N>;
  constexpr int SMEM = EPB * L::PER_ELEM;
  cudaError_t e = allow_smem(curved_volume_kernel<N, VF, EPB>, SMEM);
  if (e != cudaSuccess) return e;
  // the largest shared-memory carveout, so that the shared memory of the
  // CTAs that the registers allow fits on one SM
  e = cudaFuncSetAttribute(curved_volume_kernel<N, VF, EPB>,
                           cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  const long long grid = (g.nelem + EPB - 1) / EPB;
  curved_volume_kernel<N, VF, EPB><<<(unsigned)grid, EPB * L::LINES, SMEM, st>>>(
      u, du, fs, Ja, invJ, X, g, tb, err, fz, src);
  return cudaGetLastError();
}

// A CTA's FP64 work runs on one SM, whose FP64 pipe retires 2 lanes per
// clock: meshes with fewer elements than about two CTAs per SM run the
// pair-parallel kernel (one element per CTA, one thread per line pair),
// which shortens each thread's chain of FP64 work.
template <int N, int VF>
cudaError_t volume_n(double* u, double* du, const double* fs, const double* Ja,
                     const double* invJ, const double* X, const Geom& g, const CTables& tb,
                     unsigned* err, cudaStream_t st, const StageFuse& fz, const SourceArgs& src) {
  using L = CLaunch<N>;
  if (g.nelem < 2LL * 152 * L::EPB) {
    using C = CPairs<N>;
    cudaError_t e = allow_smem(curved_volume_pp_kernel<N, VF>, C::SMEM);
    if (e != cudaSuccess) return e;
    curved_volume_pp_kernel<N, VF><<<(unsigned)g.nelem, C::THREADS, C::SMEM, st>>>(
        u, du, fs, Ja, invJ, X, g, tb, err, fz, src);
    return cudaGetLastError();
  }
  return volume_epb<N, VF, L::EPB>(u, du, fs, Ja, invJ, X, g, tb, err, st, fz, src);
}

template <int N>
cudaError_t rhs_n(double* u, double* du, double* fs, const double* Ja, const double* invJ,
                  const double* X, const Geom& g, const CTables& tb, int vf, int sf,
                  unsigned* err, cudaStream_t st, int parts, const StageFuse& fz,
                  const SourceArgs& src) {
  if (parts & 1) {
    constexpr int NF = (N + 1) * (N + 1);
    // small meshes: 64-thread blocks, so that the face nodes reach more SMs
    const int threads = (g.nelem * NF < 152LL * 4 * 256) ? 64 : 256;
    long long blocks = (g.nelem * NF + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    curved_surface_kernel<N><<<dim3((unsigned)blocks, 3), threads, 0, st>>>(u, fs, Ja, g, sf);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!(parts & 2)) return cudaSuccess;
  if (vf == kVRanocha) return volume_n<N, kVRanocha>(u, du, fs, Ja, invJ, X, g, tb, err, st, fz, src);
  if (vf == kVChandrashekar)
    return volume_n<N, kVChandrashekar>(u, du, fs, Ja, invJ, X, g, tb, err, st, fz, src);
  return volume_n<N, kVCentral>(u, du, fs, Ja, invJ, X, g, tb, err, st, fz, src);
}

template <int N>
cudaError_t speed_n(const double* u, const double* Ja, const double* invJ, const Geom& g,
                    unsigned long long* out, unsigned* err, double* copy_to, int grid,
                    int threads, cudaStream_t st) {
  curved_speed_kernel<N><<<grid, threads, 0, st>>>(u, Ja, invJ, g, out, err, copy_to);
  return cudaGetLastError();
}

}  // namespace

#define DG_CURVED_SWITCH(CALL)        \
  switch (N) {                        \
    case 1: return CALL(1);           \
    case 2: return CALL(2);           \
    case 3: return CALL(3);           \
    case 4: return CALL(4);           \
    case 5: return CALL(5);           \
    case 6: return CALL(6);           \
    case 7: return CALL(7);           \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t curved_geometry_launch(int N, const CGeom& cg, double* Ja, double* invJ, double* Jdet,
                                   double* X, cudaStream_t st) {
#define G(n) geometry_n<n>(cg, Ja, invJ, Jdet, X, st)
  DG_CURVED_SWITCH(G)
#undef G
}

cudaError_t curved_rhs_launch(int N, double* u, double* du, double* fs, const double* Ja,
                              const double* invJ, const double* X, const Geom& g,
                              const CTables& tb, int vf, int sf, unsigned* err, cudaStream_t st,
                              int parts, const StageFuse& fz, const SourceArgs& src) {
#define R(n) rhs_n<n>(u, du, fs, Ja, invJ, X, g, tb, vf, sf, err, st, parts, fz, src)
  DG_CURVED_SWITCH(R)
#undef R
}

cudaError_t curved_speed_launch(int N, const double* u, const double* Ja, const double* invJ,
                                const Geom& g, unsigned long long* out, unsigned* err,
                                double* copy_to, int grid, int threads, cudaStream_t st) {
#define S(n) speed_n<n>(u, Ja, invJ, g, out, err, copy_to, grid, threads, st)
  DG_CURVED_SWITCH(S)
#undef S
}

}  // namespace dg
