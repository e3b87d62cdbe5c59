"""GB300-native FFT-based Zernike moments (arXiv 2304.14492).

The compute path is the C-ABI library ``libzm.so`` built from ``csrc/`` for
sm_103a; ``native`` is its thin ctypes binding.  Importing this package does
not load the library; ``native.lib()`` does, and raises if it is missing.
"""
