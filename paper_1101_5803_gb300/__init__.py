"""GB300-native semilinear lens-inversion inner loop (Rogers & Fiege 2011).

``binding``    ctypes marshalling of the C ABI in include/mirage.h
``build``      nvcc build of libmirage.so (sm_103a)
``problems``   device-resident problem sets for the five workloads
``ga``         host genetic algorithm around the batched evaluator
``surrogate``  MLP surrogate (BF16 kernels) for screening and warm starts
"""
