"""B300-native fused Lloyd k-means: a C-ABI CUDA library (include/kmeans.h) and its
Python binding. ``from paper_1109_0778_b300 import kmeans`` loads libkmeans.so and
fails loudly if it has not been built (paper_1109_0778_b300/build.py)."""
