"""GB300-native SGLD + ULISSE for Gaussian-process covariance parameters.

The compute path is the C-ABI library ``libulisse.so`` (hand-written CUDA for sm_103a),
declared in ``include/ulisse.h``.  ``paper_1501_05427_gb300.ulisse`` is the thin Python
binding (argument marshalling only); ``workloads`` makes seeded synthetic inputs.
Importing the package does not load the CUDA library; ``ulisse.load()`` does, and it raises
if the library was not built.
"""
__all__ = ["ulisse", "workloads", "build"]
