"""GB300-native orthogonalization-free Kohn-Sham total-energy minimization (PCAL).

Layout:
  inputs    seeded synthetic systems and graded P2 tetrahedral meshes (no method arithmetic)
  ofks      ctypes binding of the C-ABI library ``libofks.so`` (names mirror ``include/ofks.h``)
  build     compiles ``csrc/*.cu`` for sm_103a into ``libofks.so`` in this directory

Importing the package imports nothing else: ``inputs`` must stay usable by the CPU oracle
without touching the CUDA path.
"""
