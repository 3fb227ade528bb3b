"""GB300-native polar-coordinate discrete-Boltzmann detonation update.

The compute path is the CUDA library ``libdbm.so`` (sm_103a) behind the C ABI
declared in ``include/dbm.h``; :mod:`paper_1308_0653_gb300.dbm` is its thin
ctypes binding.  Importing the package loads nothing: the library is opened on
first use and a missing library is an error, never a fallback.
"""
__all__ = ["workloads"]
