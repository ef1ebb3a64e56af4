"""GB300-native Barabasi-Albert edge generation (Sanders & Schulz, arXiv:1602.07106).

The CUDA library ``libba.so`` (C ABI in ``include/ba.h``) does all the work; the module
``paper_1602_07106_gb300.ba`` is its thin Python binding and raises on import when the
library has not been built.  ``paper_1602_07106_gb300.workloads`` holds the seeded
synthetic inputs and does not load the library.
"""
