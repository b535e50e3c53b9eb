"""B300-native batched HeSP scheduling-partitioning simulator (arXiv 1602.05510).

The compute path lives in the CUDA library ``libhesp.so`` (C ABI declared in
``include/hesp.h``); ``paper_1602_05510_b300.hesp`` is its thin ctypes binding.
Importing this package does not load the library; the binding loads it on
first use and raises if it is missing (there is no CPU fallback).
"""
__all__ = ["workloads", "hesp"]
