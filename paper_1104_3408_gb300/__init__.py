"""GB300 (sm_103a) implementation of the CFF / Yn-filter pseudospectral shell
method (Bruegmann, arXiv:1104.3408): a C-ABI CUDA library (csrc/, built into
_lib/libcffyn.so) and its ctypes binding (cffyn.py).  PyTorch supplies device
memory and streams only."""

from . import cffyn  # noqa: F401
