"""GB300-native adaptive solver of A X = B (Sanderson & Curtin, arXiv 2007.11208).

The solver lives in libasolve.so (CUDA for sm_103a, C ABI in include/asolve.h);
``asolve`` is its ctypes binding, ``build`` compiles it, ``synth`` generates
seeded test inputs.
"""
