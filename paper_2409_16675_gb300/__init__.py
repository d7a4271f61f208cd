"""GB300-native homomorphic linear layers of CryptoTrain (arXiv 2409.16675).

The compute path is libcryptotrain.so (CUDA for sm_103a, C ABI declared in
include/cryptotrain.h).  ``native`` is its ctypes binding, ``layer`` composes
the CryptoTrain-P linear layer from it, ``workloads`` holds the seeded
synthetic inputs.  Submodules are imported on demand so that the input
generators can be used without a GPU.
"""
