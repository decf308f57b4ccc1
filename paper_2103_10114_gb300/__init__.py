"""GB300-native leap-format dynamical-core step (arXiv 2103.10114, AGCM-3DLF).

The compute path is ``libagcm.so`` (CUDA, sm_103a) behind the C ABI declared in
``include/agcm.h``; :mod:`.agcm` is the thin ctypes binding with the same names.
Importing this package loads nothing native; the library loads on first use and
raises if it has not been built.
"""
