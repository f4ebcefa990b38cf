"""GB300-native delayed approximate matrix assembly multigrid (arXiv 2005.03606).

The compute path is the CUDA library ``libmg.so`` (built from ``csrc/``) behind
the C ABI declared in ``include/mg.h``; ``paper_2005_03606_gb300.mg`` is its thin
ctypes binding.  ``paper_2005_03606_gb300.inputs`` draws seeded synthetic inputs.
Submodules are imported lazily so that the input generators work without a GPU.
"""
__all__ = ["inputs", "mg"]
