"""GB300-native Slice-within-Gibbs nested sampler for compact-binary inference.

The compute path is the C-ABI library ``libswig.so`` built from ``csrc/``
(hand-written sm_103a CUDA); ``swig`` is its thin ctypes binding.
"""
