"""GB300-native Many-Configuration Markov-Chain Monte Carlo on the SK spin glass.

The sampler runs in hand-written CUDA kernels for sm_103a behind a C ABI
(include/sk_mcmcmc.h); this package holds the build step, the thin ctypes
binding to that library and the seeded input generators.
"""
__all__ = ["inputs"]
