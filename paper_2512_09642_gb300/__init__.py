"""GB300-native Chebyshev-basis s-step CG with Forward Gauss-Seidel Gram solves
(arXiv 2512.09642), as a CUDA library with a C ABI (include/sstep_cg.h).

Submodules:
  build   compiles csrc/*.cu for sm_103a into libsstep_cg.so (in-tree)
  abi     ctypes binding with the C entry points' names (marshalling only)
  solver  SStepCG: a handle over a torch-resident CSR matrix or stencil

The library is loaded on first use of `abi`/`solver`; without it those imports raise.
"""
import importlib

__all__ = ["build", "abi", "solver", "SStepCG"]


def __getattr__(name):
    if name in ("abi", "solver", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    if name == "SStepCG":
        return importlib.import_module(f"{__name__}.solver").SStepCG
    raise AttributeError(name)
