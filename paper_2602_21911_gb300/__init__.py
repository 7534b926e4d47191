"""GB300-native (sm_103a) hot path of the FV+GRPrec ADER scheme (arXiv 2602.21911).

Modules (imported lazily, nothing loads at package import):
  grprec  -- ctypes binding of the C-ABI library libgrprec.so (include/grprec.h)
  build   -- nvcc build of libgrprec.so
  inputs  -- seeded synthetic initial data of the paper's workloads
"""
__all__ = ["grprec", "build", "inputs"]
