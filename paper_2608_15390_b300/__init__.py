"""B300-native (sm_103a) estimator of sparse-matrix permanents: the adaptive
sequential importance sampler of "The Quick and the Dead" (Algorithm 2) as
hand-written CUDA behind the C ABI of include/pm.h.

``binding`` (the ctypes layer) is imported on demand so that the input
generators in ``inputs`` stay usable on machines without the built library.
"""
__all__ = ["inputs", "binding", "build"]
