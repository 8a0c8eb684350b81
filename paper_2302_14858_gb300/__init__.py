"""GB300-native compact finite-difference operators (arXiv 2302.14858 hot path).

The compute path is the C-ABI shared library built from ``csrc/`` (hand-written
sm_103a CUDA); ``cfd`` is its thin Python binding.  ``workloads`` generates
seeded synthetic inputs and MeshBlock layouts.
"""
