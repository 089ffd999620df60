"""GB300-native engine for the stationary timestamp pmf of asynchronous
single-photon LiDAR under dead time (arXiv 2509.20500).

The compute path is the C-ABI library ``libspl`` (hand-written sm_103a CUDA),
declared in ``include/spl.h``; ``paper_2509_20500_gb300.spl`` is its thin
ctypes binding.  Importing this package loads nothing; the library is loaded
on first use of the binding and a missing library raises.
"""
__all__ = ["spl", "workloads"]
