"""RIANN per-frame query engine for NVIDIA GB300 (sm_103a).

The compute path lives in ``csrc/`` (CUDA kernels behind the C ABI of
``include/riann.h``) and is reached through :mod:`paper_1508_07953_gb300.riann`,
a ctypes binding with the same names as the C entry points.  Importing this
package loads nothing; ``riann`` fails loudly if the library was not built.
"""
