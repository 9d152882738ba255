"""GB300-native Johnson-Lindenstrauss sketching for adaptive HSS construction.

* ``jlsketch``  -- ctypes binding of libjlsketch (include/jlsketch.h): the C ABI
  whose CUDA kernels compute S = A R and S' = A^T R for SJLT, SRHT and
  Gaussian operators, grow R by increments and run the stopping test.
* ``inputs``    -- seeded synthetic points and matrices (no sketch arithmetic).
* ``build``     -- nvcc build of the shared library for sm_103a.

Nothing is imported eagerly, so ``inputs`` can be used without the library.
"""
