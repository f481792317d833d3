"""GB300-native adaptive TT cross (arXiv 2407.11290): Python binding.

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI declared in
``include/ttcross.h``); this package only loads that library and marshals
arguments.  Importing the package does not load the library: the first call
into :mod:`paper_2407_11290_gb300.ttcross` does, and raises if it is missing.
"""
__all__ = ["ttcross", "workloads"]
