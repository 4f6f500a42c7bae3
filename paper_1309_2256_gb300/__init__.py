"""GB300 (sm_103a) disconnected-quark-loop library: the even-odd twisted-mass
solver, Z4 noise, loop contractions and the Truncated Solver Method behind the C
ABI of include/discloop.h.  This package is the Python binding of that ABI; all
computation runs in the CUDA kernels of libdiscloop.so."""
from ._binding import *  # noqa: F401,F403
from ._binding import lib, DLError  # noqa: F401
