"""GB300-native free-surface lattice Boltzmann step (arXiv 2207.14496).

The compute path is the CUDA library ``libfsl`` (C ABI declared in
``include/fsl.h``); ``paper_2207_14496_gb300.fsl`` is its thin Python binding.
Importing the package does not load the library; ``fsl`` does, and raises if
the compiled library is missing.
"""
__all__ = ["inputs"]
