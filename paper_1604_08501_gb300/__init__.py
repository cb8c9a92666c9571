"""GB300-native (sm_103a) element volume term of a NUMA-style compressible
Euler model on hexahedral GLL spectral elements (Kloeckner, Wilcox,
Warburton, ARRAY'16, Sec. 2, Eq. (2)).

Submodules:
  numa_vol  -- Python binding of the C ABI (VolumeTerm, diff_matrix)
  workload  -- seeded synthetic meshes, reference states and states
  build     -- in-tree nvcc build of libnumavol.so

Importing the package loads no native code.  The CUDA library is loaded on
first use and raises if it has not been built.
"""

__all__ = ["numa_vol", "workload", "build"]
