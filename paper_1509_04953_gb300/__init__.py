"""GB300-native (sm_103a) coupled FFT-EVP / phase-field DRX hot path (arXiv:1509.04953).

The compute path lives in the CUDA library libevp_gb300.so behind the C ABI declared in
include/evp.h; `paper_1509_04953_gb300.evp` is its thin ctypes binding. Importing this package
does not load the library; the binding loads it on first use and raises if it is missing.
"""
__all__ = ["synth", "evp"]
