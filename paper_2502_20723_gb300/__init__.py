"""GB300-native transformer density-operator ansatz: batched log rho, local estimator,
Metropolis sampling, log-derivatives and stochastic reconfiguration, all in CUDA kernels
for sm_103a behind the C ABI declared in include/tdo.h.

Importing the package loads nothing; ``paper_2502_20723_gb300.tdo`` loads libtdo.so and
raises if it is missing (there is no CPU fallback).
"""
__all__ = ["synth"]
