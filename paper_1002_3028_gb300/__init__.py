"""GB300-native axisymmetric thermal lattice Boltzmann LES (arXiv:1002.3028).

The compute path is the C-ABI library ``liblbm`` (hand-written CUDA for
sm_103a); :mod:`paper_1002_3028_gb300.lbm` is its thin Python binding.
"""
