"""GB300-native (sm_103a) electromagnetic particle-in-cell hot path.

The compute path is the C-ABI library libpic (CUDA kernels in csrc/, API in
include/pic.h); `paper_2101_12149_gb300.pic` is its thin ctypes binding.
`paper_2101_12149_gb300.inputs` holds the seeded synthetic workload
generators.  Importing the package loads nothing; the binding loads libpic on
first use and fails loudly if it is missing.
"""
__all__ = ["inputs", "pic"]
