"""GB300 implementation of one Strang step of the CHASM scheme for 6-D Wigner-Coulomb dynamics
(Xiong, Zhang, Shao, arXiv 2205.02380): CUDA kernels behind the C ABI of include/chasm.h, with a
ctypes binding in ``chasm``."""
from . import chasm  # noqa: F401
from .chasm import (FP32_MIXED, FP64, LPC1, STRANG, THETA_AUTO, THETA_MODULATED,  # noqa: F401
                    THETA_TABLE,
                    ChasmError, Server, Solver, make_request)
