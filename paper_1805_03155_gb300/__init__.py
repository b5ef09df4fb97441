"""GB300-native SPSTD solver (arXiv 1805.03155): C-ABI library + thin binding.

Importing the package loads nothing; ``paper_1805_03155_gb300.spstd`` loads the
CUDA library on first use and raises if it is missing.
"""
