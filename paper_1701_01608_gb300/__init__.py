"""GB300-native Fast Kinetic Scheme hot path (arXiv 1701.01608).

The compute path is the CUDA library ``csrc/`` built into ``libfks.so``;
``fks`` is its thin ctypes binding.  Importing this package does not load
the library; ``paper_1701_01608_gb300.fks`` does.
"""
