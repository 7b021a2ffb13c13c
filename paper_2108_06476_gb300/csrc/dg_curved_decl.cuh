// Curvilinear-mesh parameters shared by the kernels (dg_curved.cuh) and the
// C ABI (dg_api.cu), and the host-side launchers of dg_curved.cu.
#pragma once
#include "dg_device.cuh"

namespace dg {

struct CGeom {
  Geom g;
  double warp;                       // amplitude of the warping (0.15 in the paper)
  double xi[kNPMax];                 // LGL nodes
  double D[kNPMax][kNPMax];          // nodal derivative matrix
  const double* Xin;                 // given node coordinates [e][3][P] (nullptr: the warp)
};

// split form with the sign of du folded in: Ds = -Dt, liftR = -1/w_N,
// liftL = 1/w_0 (du = (1/J) acc + S)
struct CTables {
  double Ds[kNPMax][kNPMax];
  double liftR, liftL;
};

// manufactured-solution source term: rho = 2 + A sin(pi (x + y + z - t)),
// v = (1, 1, 1), E = rho^2, A = 0.1; time t = *t0 + c * (*dt) (dt may be
// null: t = *t0)
enum { kSourceNone = 0, kSourceManufactured = 1 };
struct SourceArgs {
  int kind = kSourceNone;
  const double* t0 = nullptr;
  const double* dt = nullptr;
  double c = 0.0;
};

// host-side entry points (dg_curved.cu)
cudaError_t curved_geometry_launch(int N, const CGeom& cg, double* Ja, double* invJ, double* Jdet,
                                   double* X, cudaStream_t st);
// parts: 1 surface, 2 volume, 3 both (as the Cartesian launcher)
cudaError_t curved_rhs_launch(int N, double* u, double* du, double* fs, const double* Ja,
                              const double* invJ, const double* X, const Geom& g,
                              const CTables& tb, int vf, int sf, unsigned* err, cudaStream_t st,
                              int parts, const StageFuse& fz, const SourceArgs& src);
cudaError_t curved_speed_launch(int N, const double* u, const double* Ja, const double* invJ,
                                const Geom& g, unsigned long long* out, unsigned* err,
                                double* copy_to, int grid, int threads, cudaStream_t st);

}  // namespace dg
