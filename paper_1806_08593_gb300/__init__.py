"""GB300-native Tensor Monte Carlo hot path (Aitchison, "Tensor Monte Carlo: Particle
Methods for the GPU Era", ICML 2019).

Submodules:
    workload  seeded synthetic linear-Gaussian chains / trees (numpy only)
    tmc       C-ABI binding (ctypes) and the torch.autograd.Function wrapper
"""
__all__ = ["workload", "tmc"]
