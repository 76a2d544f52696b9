"""GB300 (sm_103a) implementation of the BSGD-TV hot path (arXiv 1812.01307).

Modules:
  bsgdtv  -- ctypes binding of the C ABI in include/bsgdtv.h (libbsgdtv.so)
  build   -- nvcc build of libbsgdtv.so
  synth   -- seeded synthetic inputs (phantom, Siddon projector, noise)
Nothing is imported here, so ``synth`` can be used without the CUDA library.
"""
