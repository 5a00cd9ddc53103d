"""GB300-native structure-preserving reduction of Yee FDTD equations.

The compute path lives in the CUDA library ``libfdtdmor.so`` (C ABI declared in
``include/fdtdmor.h``); ``paper_1406_7042_gb300.fdtdmor`` is its thin ctypes
binding.  ``workloads`` builds the seeded synthetic inputs.  Importing the
package does not load the CUDA library; the binding loads it on first use and
raises if it is missing.
"""
__all__ = ["workloads"]
