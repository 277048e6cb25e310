"""GB300-native Parallel Toplesets Propagation (PTP) geodesic distances.

The computation lives in the CUDA library libptp.so (C ABI in include/ptp.h);
`capi` is its thin Python binding and `meshes` generates seeded synthetic
inputs.  Importing this package loads nothing; the library is loaded on the
first call and the call fails loudly if it has not been built.
"""
