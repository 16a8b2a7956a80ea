"""B300-native batched MD5 / SHA-1 / SM3 hashing.

The compute path is the CUDA library ``libhashbatch.so`` built from ``csrc/``
for sm_103a; ``api`` is a thin ctypes binding over its C-ABI (declared in
``include/hashbatch.h``).  ``workloads`` draws the seeded synthetic inputs.
Submodules are imported explicitly (``from paper_2407_09333_b300 import api``).
"""
