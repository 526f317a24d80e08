"""GB300 (sm_103a) implementation of the TT-ICE / TT-ICE* incremental tensor-train update.

The library is ``libttice.so`` (C ABI in include/ttice.h, CUDA kernels in csrc/); ``ttice`` is its
Python binding.  Import ``paper_2211_12487_gb300.ttice`` after building with
``paper_2211_12487_gb300.build.build()``.
"""
