"""GB300-native spiking-network simulator core (LIF exact integration, AdEx
adaptive RK45, delay-grouped CSR spike delivery) behind the C ABI in
include/ngb.h.

Importing the package does not load the CUDA library; ``from
paper_2007_14236_gb300 import ngb`` does, and fails loudly if it is missing.
"""
__all__ = ["workloads"]
