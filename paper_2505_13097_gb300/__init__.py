"""GB300 implementation of the implicit regularized enthalpy lattice Boltzmann
method (IREBM) for the Stefan problem (Luddens, Lothode, Danaila, arXiv 2505.13097).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbm_stefan.h``); ``solver`` and ``autograd`` marshal arguments into
it.  ``workloads`` holds the seeded synthetic inputs.
"""
from ._abi import (LBM_ADIABATIC, LBM_BB_LINK, LBM_BB_MIRROR, LBM_D1Q3, LBM_D2Q9, LBM_DIRICHLET, LBM_FP32,
                   LBM_FP64, LBMError)

__all__ = ["LBM_ADIABATIC", "LBM_BB_LINK", "LBM_BB_MIRROR", "LBM_D1Q3", "LBM_D2Q9", "LBM_DIRICHLET",
           "LBM_FP32", "LBM_FP64", "LBMError"]
