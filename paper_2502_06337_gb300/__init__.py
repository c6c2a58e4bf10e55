"""GB300-native stereographic-projection rotation vote (arXiv 2502.06337).

The compute path lives in the CUDA library ``libsprot.so`` (sources in ``csrc/``, C ABI in
``include/sprot.h``); ``binding`` is a thin ctypes layer over it. ``synth`` draws seeded
synthetic problems. Importing the package does not load the library.
"""
