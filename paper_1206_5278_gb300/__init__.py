"""GB300 (sm_103a) library for exact leave-one-out bandwidth selection of the
double-kernel conditional density estimator (Holmes, Gray & Isbell,
"Fast Nonparametric Conditional Density Estimation").

The compute path is ``libcde.so`` (hand-written CUDA kernels behind the C ABI
of ``include/cde.h``); ``cde`` is its ctypes binding.  Importing this package
does not load the library; ``cde.lib()`` does, and fails loudly when it is
missing.
"""
__all__ = ["cde", "synth"]
