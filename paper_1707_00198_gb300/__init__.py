"""GB300-native colour-gradient lattice Boltzmann with the improved geometric wetting
scheme of arXiv 1707.00198.  The compute path is the CUDA library ``liblbcg.so`` (built
from ``csrc/``); ``lbcg`` is its ctypes binding and ``inputs`` holds the seeded synthetic
workloads."""
