"""GB300-native Contour-FFT (C-FFT) tabulation of MBF reaction terms.

The compute path is the CUDA library ``libcfft.so`` (sm_103a), reached through
the C ABI of ``include/cfft.h``; ``paper_1404_7357_gb300.cfft`` is a thin ctypes
binding with the same call names.  Nothing in this package computes the
method on the CPU: if the library is missing, importing the binding raises.
"""
