"""GB300-native finite-difference acoustic wave propagation (arXiv 1609.03361 hot path).

The compute path is the CUDA library ``libfdwave.so`` (C ABI, ``include/fdwave.h``);
``paper_1609_03361_gb300.fdwave`` is its thin Python binding.
"""
