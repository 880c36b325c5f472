"""GB300-native CTMRG in the Hermitian (bra-ket swap) basis of arXiv 2410.11596.

The compute path is the CUDA library libhs.so (C ABI in include/hs.h), built
in-tree by ``paper_2410_11596_gb300.build``. ``_lib`` is its ctypes binding and
``api`` a thin front end that allocates device buffers with torch. Importing
this package does not load the library; ``_lib.load()`` does, and fails if the
library is missing.
"""
