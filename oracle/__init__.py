"""Plain FP64 CPU oracle for the Krylov-vector evaluation (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package. The CUDA product path never does.
"""
from .oracle import Oracle, build_oracle  # noqa: F401
