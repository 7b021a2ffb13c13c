// Instantiates the rhs kernels for one arithmetic type and one dimension.
// Compiled once per (DG_INST_REAL, DG_INST_DIM) pair so that the template
// instantiations build in parallel translation units.
#include "dg_rhs_kernels.cuh"

#ifndef DG_INST_REAL
#error "define DG_INST_REAL (double or float)"
#endif
#ifndef DG_INST_DIM
#error "define DG_INST_DIM (2 or 3)"
#endif

#define DG_CAT2(a, b, c) a##_##b##_##c
#define DG_CAT(a, b, c) DG_CAT2(a, b, c)

namespace dg {
cudaError_t DG_CAT(rhs_launch, DG_INST_REAL, DG_INST_DIM)(int N, const double* u, DG_INST_REAL* du,
                                                          DG_INST_REAL* fs, const Geom& g,
                                                          const Tables<DG_INST_REAL>& tb, int vf,
                                                          int sf, unsigned* err, cudaStream_t st,
                                                          int parts, const StageFuse& fz) {
  return launch_rhs_d<DG_INST_DIM, DG_INST_REAL>(N, u, du, fs, g, tb, vf, sf, err, st, parts, fz);
}
}  // namespace dg
