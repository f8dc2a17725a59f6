"""RotorMap hot path on GB300 (sm_103a): C-ABI CUDA library + thin binding.

``rotormap`` holds the binding (same names as include/rotormap.h); ``build``
compiles ``librotormap.so`` in-tree.
"""
