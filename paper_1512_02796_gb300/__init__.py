"""GB300 (sm_103a) hot path of QPAT reconstruction with total-variation-type
priors: matrix-free P1 diffusion operators, persistent fused PCG, matrix-free
Jacobian products, lagged-diffusivity prior solves and priorconditioned LSQR,
behind the C ABI of include/qpat.h (libqpat.so).  `qpat` is the Python
binding of that ABI."""
from . import qpat  # noqa: F401
from .qpat import *  # noqa: F401,F403
