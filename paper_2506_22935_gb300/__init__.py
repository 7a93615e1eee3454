"""GB300-native differentiable radar ambiguity function (AF).

``graf``   - ctypes binding of libgraf.so (C ABI in include/graf.h) and torch
             conveniences; every computation runs in the library's kernels.
``inputs`` - seeded synthetic inputs (no method arithmetic).
``_build`` - builds libgraf.so for sm_103a.
"""
