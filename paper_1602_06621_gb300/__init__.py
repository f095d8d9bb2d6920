"""GB300 (sm_103a) stochastic matrix-free equilibration (Diamond & Boyd).

The compute path is libsme.so, a C-ABI CUDA library (include/sme.h); `sme` is its
thin ctypes binding.  Importing this package loads nothing: the library is built
and loaded on first use of `paper_1602_06621_gb300.sme`.
"""
