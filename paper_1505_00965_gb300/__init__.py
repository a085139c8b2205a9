"""GB300-native multilevel Monte Carlo level engine (sm_103a).

* ``paper_1505_00965_gb300.mlmc``  -- Python binding of the C ABI in include/mlmc.h (the CUDA
  library must be built; importing the binding fails loudly otherwise).
* ``paper_1505_00965_gb300.build`` -- in-tree build of ``libmlmc_gb300.so`` with nvcc.
"""
