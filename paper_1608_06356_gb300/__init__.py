"""GB300-native per-macroparticle QED Monte Carlo step (arXiv:1608.06356).

The compute path is libqed.so (CUDA kernels for sm_103a behind the C ABI of
include/qed.h); ``api`` wraps it for torch tensors, ``workloads`` holds the
seeded synthetic input generators, and ``build`` compiles the library.
Importing this package does not load the library; the first call does, and
raises if it has not been built.
"""
from .build import build  # noqa: F401

__all__ = ["build", "api", "workloads"]
