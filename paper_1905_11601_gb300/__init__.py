"""GB300 (sm_103a) Krylov-vector evaluation for the stability of natural convection in a
laterally heated cube (Gelfgat, arXiv 1905.11601, Section 3.1).

``kv`` is the Python binding of libkv.so (include/kv.h); ``synth`` draws the seeded synthetic
inputs; ``build`` compiles the CUDA library in-tree.
"""
from . import synth  # noqa: F401
