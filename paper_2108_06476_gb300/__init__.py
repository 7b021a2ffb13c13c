"""GB300-native DGSEM for the 2D/3D compressible Euler equations.

Hot path: the split-form (entropy-conservative flux differencing) DGSEM
right-hand side on a uniform periodic Cartesian mesh and the Carpenter-Kennedy
low-storage RK stage, as hand-written CUDA kernels for sm_103a behind the C
ABI in include/dgsem.h. This package holds the in-tree build script, the
ctypes binding and the seeded workload generators.
"""
from .dgsem import (Mesh, Ensemble, MeshSpec, DGError, lgl_nodes, load, measure_peaks,  # noqa: F401
                    measure_fp64_issue, RK_A, RK_B, SO_PATH)
from . import workloads  # noqa: F401
