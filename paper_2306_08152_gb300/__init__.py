"""GB300-native QFactor instantiation engine.

QFactor (Kukliansky, Younis, Cincio, Iancu, arXiv 2306.08152) fits a circuit
of general two-qubit unitaries to a target unitary by sweeping one circuit
tensor.  The sweep runs in hand-written CUDA kernels for sm_103a behind the
C ABI of include/qfactor.h; this package is the thin Python binding.
"""
from .api import *  # noqa: F401,F403
from .api import __all__  # noqa: F401
from . import _native  # noqa: F401
from ._native import QFactorError  # noqa: F401
from .autograd import QFactorCost, qfactor_cost  # noqa: F401
