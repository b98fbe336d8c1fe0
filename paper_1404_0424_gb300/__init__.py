"""GB300-native CG soft-output MMSE detection and CG precoding.

The compute path is the C-ABI library libcgmimo.so (hand-written sm_103a
CUDA). Importing this package does not load it; `paper_1404_0424_gb300.cabi`
loads it on first use and raises if it is missing.
"""

__all__ = ["cabi", "workload"]
