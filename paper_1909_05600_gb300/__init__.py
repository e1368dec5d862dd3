"""GB300-native hot path of the Fast Free Memory method (arXiv:1909.05600).

The compute path is the CUDA library `libffm_gb300.so` (sm_103a), reached through the
C ABI declared in include/ffm.h.  `paper_1909_05600_gb300.ffm` holds the thin Python
binding; `workloads` holds the seeded synthetic inputs.  Importing this package loads
nothing: the library is opened on first use and fails loudly if it is missing.
"""
__version__ = "0.1.0"
