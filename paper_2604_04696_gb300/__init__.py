"""GB300-native RowSel (GPIR, arXiv 2604.04696): C-ABI library + thin binding.

Importing the package does not load CUDA; ``paper_2604_04696_gb300.gpir`` loads
libgpir.so (and raises if it is missing) and ``.server`` holds the serving loop.
"""

__version__ = "0.1.0"
