"""GB300-native (sm_103a) high-order finite-volume JFNK library for solid
mechanics (Batistic, Castrillo & Cardiff, arXiv 2601.18417).

The compute path lives in ``libhofv.so`` (CUDA + C++, C ABI declared in
``include/hofv.h``); ``paper_2601_18417_gb300.hofv`` is the thin Python
binding over it.  ``paper_2601_18417_gb300.inputs`` holds the seeded
synthetic workloads.  Importing the package does not load the CUDA library;
the first call into ``hofv`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs", "hofv"]
