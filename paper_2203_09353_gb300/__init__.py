"""GB300-native batched small-GEMM library (Eq. 1 of the paper, Sec. 2)."""
