"""GB300-native Building Cube Method (BCM) time step: C-ABI CUDA library + Python binding."""
