"""GB300-native MOL^T recursive-convolution wave solver (arXiv:1308.3214).

The compute path is the CUDA library ``libmolt.so`` (C ABI declared in
``include/molt.h``); ``paper_1308_3214_gb300.molt`` is its thin ctypes binding.
"""
