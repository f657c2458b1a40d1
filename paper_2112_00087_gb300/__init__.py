"""GB300-native frequency-response solver for the cavity Helmholtz problem.

The compute path is the CUDA library libhelm.so (C ABI in include/helm.h); `helm` is its
ctypes binding. Importing the binding loads the library and raises if it was not built.
"""
__all__ = ["helm"]
