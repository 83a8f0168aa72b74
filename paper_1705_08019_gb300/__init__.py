"""GB300-native FIT leapfrog + ParaExp (Merkel, Niyonzima, Schoeps).

The compute path is libfitgb.so (hand-written CUDA for sm_103a) behind the C
ABI declared in include/fitgb.h; ``paper_1705_08019_gb300.fitgb`` is its
ctypes binding and ``paper_1705_08019_gb300.workloads`` the seeded synthetic
inputs.  ``paper_1705_08019_gb300.build`` compiles the library in-tree.
"""
