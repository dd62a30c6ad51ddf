"""GB300 (sm_103a) charge-readout hot path of the pixelated LArTPC simulation of
arXiv:2212.09807: recombination, drift, pixel mapping, induced current and
front-end electronics as CUDA kernels behind the C ABI of include/sim.h.

``sim`` is the ctypes binding; ``build`` compiles ``libsim.so`` in-tree.
"""
