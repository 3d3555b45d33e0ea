"""GB300-native LocalContraction connected components (arXiv 1807.10727).

The compute path is the CUDA library ``_lib/liblc.so`` behind the C ABI in
``include/lc.h``; :mod:`paper_1807_10727_gb300.lc` is its thin ctypes binding.
"""
