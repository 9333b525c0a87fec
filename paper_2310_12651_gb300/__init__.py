"""GB300-native fast force-coupling method: the periodic mobility product (U, W) = M (F, T).

The compute path is the C-ABI library ``libfcm`` (hand-written sm_103a CUDA plus
cuFFT for the transforms); ``paper_2310_12651_gb300.fcm`` is its thin ctypes
binding. Importing this package loads nothing: the library is opened on first
use of the binding, and the binding raises if the compiled library is missing.
"""
