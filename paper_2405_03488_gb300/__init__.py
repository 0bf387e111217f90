"""GB300-native approximate graph pattern mining (neighbour sampling with eager
verify, online convergence detection, colour sparsification, hybrid choice).

The compute path is libgpm.so (CUDA, sm_103a) behind the C ABI in
include/gpm.h; ``api`` wraps it for PyTorch tensors and streams.
"""
