"""GB300-native coupled LBM-PSM-DEM time step (LEDDS, arXiv 2512.04997).

Submodules:
  ``ledds``      ctypes binding of the C-ABI library ``libledds.so`` (include/ledds.h)
  ``workloads``  seeded synthetic inputs shaped like the paper's runs
  ``build``      nvcc build step of the CUDA library
The package imports nothing heavy at import time; the binding loads the CUDA library on
first use and raises if it is missing.
"""
__all__ = ["ledds", "workloads", "build"]
