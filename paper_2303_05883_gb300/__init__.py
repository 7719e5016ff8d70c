"""GB300 (sm_103a) implementation of the Wilson/clover fermion-solver path.

The even-odd preconditioned Wilson/clover Dirac operator (Eq. 1) inside a
mixed-precision BiCGStab with FP64 defect correction, multi-right-hand-side
batching and a continuous-batching request engine.  The work runs in the
hand-written CUDA kernels of ``libbridge.so`` (C-ABI in include/bridge.h);
this package is its ctypes binding and the in-tree build.
"""

from ._abi import load  # noqa: F401
from .api import *  # noqa: F401,F403
from .api import Lattice, make_op, make_solver  # noqa: F401
