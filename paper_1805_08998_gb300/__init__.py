"""GB300-native H-matrix product with blockwise eps-best truncation.

The CUDA library (libhmat.so, C-ABI in include/hmat.h) is loaded lazily by
``paper_1805_08998_gb300.hmat``; ``paper_1805_08998_gb300.inputs`` holds the seeded point
generator and imports nothing else.
"""

__all__ = ["hmat", "inputs", "build_lib"]
