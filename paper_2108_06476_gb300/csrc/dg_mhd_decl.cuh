// Launchers of the 3D ideal MHD kernels (dg_mhd.cu), for the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "dg_curved_decl.cuh"
#include "dg_device.cuh"

namespace dg {

// One rhs evaluation (parts: bit 0 face kernel, bit 1 volume kernel); tb
// holds Ds = -(2/h) D per direction and the lifting factors (weak form),
// tdt Ds = -(2/h) Dt (split form); vf 0 weak form, 1 entropy-conservative
// flux differencing; fs holds 3 * 9 * nelem * (N+1)^2 doubles; sf 0 LLF,
// 1 HLL, 2 EC; fz (optional) fuses the stage update.
cudaError_t mhd_rhs_launch(int N, const double* u, double* du, double* fs, const Geom& g,
                           const Tables<double>& tb, const Tables<double>& tdt, int vf,
                           int powell, int sf, unsigned* err, cudaStream_t st, int parts,
                           const StageFuse& fz);

// Wave-speed reduction sum_dir s[dir] max(|v_dir| + c_f,dir) into out (as
// ordered bits); copy_to (optional) receives a copy of u.
cudaError_t mhd_speed_launch(const double* u, const Geom& g, int P, const double* s,
                             unsigned long long* out, unsigned* err, double* copy_to, int grid,
                             int threads, cudaStream_t st);

// The same on the warped box: Ja, invJ from the curved geometry, tb the
// unscaled split-form table (Ds = -Dt, liftR = -1/w_N, liftL = 1/w_0).
cudaError_t mhd_curved_rhs_launch(int N, const double* u, double* du, double* fs, const double* Ja,
                                  const double* invJ, const Geom& g, const CTables& tb, int vf,
                                  int powell, int sf, unsigned* err, cudaStream_t st, int parts,
                                  const StageFuse& fz);

// Wave-speed reduction on the warped box: sum_r max_nodes (|v . J a^r| +
// c_f |J a^r|) / J per element, max over elements.
cudaError_t mhd_curved_speed_launch(const double* u, const double* Ja, const double* invJ,
                                    const Geom& g, int P, unsigned long long* out, unsigned* err,
                                    double* copy_to, int grid, int threads, cudaStream_t st);

}  // namespace dg
