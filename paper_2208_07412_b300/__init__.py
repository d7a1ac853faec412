"""B300-native TPC timeframe reconstruction (ZS decode, cluster finder, CA
seeding, merge, Kalman fit) behind the C ABI of include/tpc.h.

The compute path is libtpc_b300.so (hand-written sm_103a CUDA kernels); this
package only marshals arguments to it (see tpc.py).
"""
from .tpc import *  # noqa: F401,F403
from .tpc import Reconstructor, TpcError, load, library_path  # noqa: F401

__all__ = ["Reconstructor", "TpcError", "load", "library_path"]
