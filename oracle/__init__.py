"""FP64 CPU oracle for QFactor (test infrastructure only).

This package is a plain, slow, obviously-correct NumPy restatement of the
QFactor method of Kukliansky, Younis, Cincio and Iancu (Sec. III, Alg. 1,
Eq. opt_u).  It exists to check the CUDA path: only the test suite, the
package smoke check and the benchmark's CPU-baseline leg may import it.  The
product path never calls it, and it shares no code with the CUDA kernels.

Parity status of every function is stated in ``oracle/qfactor_oracle.py``.
"""
from .qfactor_oracle import *  # noqa: F401,F403
from .qfactor_oracle import __all__  # noqa: F401
