"""GB300-native (sm_103a) hot path of the multipatch scalar-wave method of
"PatchworkWave" (arXiv:2002.00088).

``paper_2002_00088_gb300.mpw`` is the ctypes binding of libmpw.so (C ABI in
include/mpw.h; importing it requires the built library);
``workloads`` holds the seeded synthetic configurations; ``build`` compiles
the CUDA library in-tree.
"""
from . import build, workloads  # noqa: F401

__all__ = ["build", "workloads"]
