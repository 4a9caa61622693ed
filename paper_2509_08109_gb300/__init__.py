"""GB300-native structured black-box multigrid (BoxMG) solver for diffusion
problems mapped onto a structured computational grid.

The solver is the CUDA library ``libbmg.so`` (sources in ``csrc/``, C ABI
declared in ``include/bmg.h``); ``binding`` wraps it with ctypes and torch
tensors.  Importing this package does not load the library; the first use
of ``binding`` does, and fails loudly if it has not been built.
"""
__all__ = ["binding", "inputs"]
