"""GB300-native lattice-Boltzmann solver for flow of mixtures through
anisotropic porous media (Mendoza, Wittel and Herrmann, arXiv:0912.4230).

The compute path is the CUDA library ``liblbgb.so`` (C ABI declared in
``include/lb.h``); :mod:`paper_0912_4230_gb300.lb` is its thin ctypes binding.
"""
