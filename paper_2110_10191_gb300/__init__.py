"""GB300-native (sm_103a) GRMHD predictor-corrector step of the HARM scheme
(iharm3D, arXiv:2110.10191) behind the C ABI of include/grmhd.h.

Submodules are imported on demand:
  build     -- nvcc build of libgrmhd.so
  grmhd     -- ctypes binding (Sim, fp64_peak)
  problems  -- seeded synthetic initial conditions
"""
