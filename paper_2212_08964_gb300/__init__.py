"""Load-balanced CSR SpMV for NVIDIA GB300 (sm_103a).

The compute path is ``liblbspmv.so`` (hand-written CUDA behind the C ABI in
``include/lbspmv.h``); ``lbspmv`` is its Python binding, ``synth`` builds seeded synthetic
inputs, and ``autotune`` picks launch shapes per matrix-shape class.
"""
__version__ = "1.0.0"
