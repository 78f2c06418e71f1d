"""GB300-native two-component Shan-Chen D2Q9 lattice Boltzmann with wetting
boundary conditions (arXiv:2009.12584).

The compute path is the CUDA library ``liblbm_gb300.so`` (C ABI declared in
``include/lbm.h``); :mod:`paper_2009_12584_gb300.lbm` is its thin ctypes
binding. Importing the package loads nothing; the library is opened on the
first call that needs it and an error is raised if it has not been built.
"""

__all__ = ["lbm", "inputs"]
