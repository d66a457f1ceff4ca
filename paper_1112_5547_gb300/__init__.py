"""GB300-native two-component Shan-Chen lattice Boltzmann step.

The compute path is the CUDA library ``liblbm_sc.so`` built from ``csrc/``
(C-ABI declared in ``include/lbm_sc.h``); ``lbm_sc`` is its thin ctypes
binding.  Submodules are imported lazily so that the input recipes can be used
without loading the CUDA library.
"""
__all__ = ["lbm_sc", "inputs", "params", "build"]
