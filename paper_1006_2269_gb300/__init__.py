"""GB300-native (sm_103a) asymmetric adaptive 2D fast multipole method.

The compute path is the CUDA library ``libfmm_gb300.so`` (C ABI declared in ``include/fmm.h``);
:mod:`paper_1006_2269_gb300.fmm` is its thin ctypes binding, with the same entry-point names.
Importing this package does not load the library; the first call into :mod:`.fmm` does, and it
raises if the library has not been built -- there is no CPU fallback.
"""
