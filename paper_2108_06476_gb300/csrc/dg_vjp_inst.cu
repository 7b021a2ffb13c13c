// Instantiates the rhs vector-Jacobian-product kernels for one arithmetic
// type and one dimension (compiled once per pair, in parallel).
#include "dg_vjp_kernels.cuh"

#define DG_CAT2(a, b, c) a##_##b##_##c
#define DG_CAT(a, b, c) DG_CAT2(a, b, c)

namespace dg {
cudaError_t DG_CAT(vjp_launch, DG_INST_REAL, DG_INST_DIM)(int N, const double* u, const double* w,
                                                          double* ubar, double* fb, const Geom& g,
                                                          const Tables<double>& tb, int vf,
                                                          int sf, cudaStream_t st) {
  return launch_vjp_d<DG_INST_DIM, DG_INST_REAL>(N, u, w, ubar, fb, g, tb, vf, sf, st);
}
}  // namespace dg
