"""GB300-native semilinear lens-inversion inner loop (Rogers & Fiege 2011).

``binding``    ctypes marshalling of the C ABI in include/mirage.h
``build``      nvcc build of libmirage.so (sm_103a)
``problems``   device-resident problem sets for the workloads
``ga``         genetic algorithm around the batched evaluator, with the MLP
               surrogate screen (BF16 kernels) and lambda chains
``pso``        particle swarm (Eq. PSO) around the batched evaluator
``refine``     positivity refinement of the source on the forward batch
``autotune``   CGLS kernel-variant tuner per shape class
"""
