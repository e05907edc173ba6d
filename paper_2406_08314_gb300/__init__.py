"""GB300-native multi-Slater-determinant AFQMC hot path (overlap, force bias,
local energy by generalized Wick's theorem), after Huang, Guo, Pham and Lv,
"GPU-accelerated auxiliary-field quantum Monte Carlo with multi-Slater
determinant trial states".

Submodules:
  synth  -- seeded synthetic systems and walkers (no method arithmetic)
  msd    -- ctypes binding of the C-ABI library libmsd.so (CUDA, sm_103a)
  build  -- compiles libmsd.so in-tree with nvcc
"""
__all__ = ["synth", "msd", "build"]
