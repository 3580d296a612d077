"""GB300-native (sm_103a) TAPS hot path: CP tensor-decomposition space-parameter-time
Galerkin solve on 1D C-HiDeNN shape functions.

The compute path is the C-ABI library ``libtaps.so`` built from ``csrc/``; the
Python module ``taps`` is a thin ctypes binding over it.  ``workloads`` holds the
seeded synthetic problem descriptions.
"""
