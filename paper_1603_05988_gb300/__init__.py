"""GB300-native deflated Hutchinson estimator of Tr(A^-1) for the Wilson-Dirac matrix.

The compute path lives in the CUDA shared library built from ``csrc/``
(``libdtr.so``, C ABI declared in ``include/dtr.h``); ``dtr`` is its thin
ctypes binding.  ``synth`` draws the seeded synthetic inputs.
"""
