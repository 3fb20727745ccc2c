"""GB300-native pyramidal Lucas-Kanade (KLT) tracking.

The compute path is libvt.so (hand-written CUDA for sm_103a behind the C ABI
of include/vt.h); ``vt`` is its ctypes binding.  Importing the package loads
the library and fails loudly if it is missing.
"""

from .vt import *  # noqa: F401,F403
from .vt import (Pyramid, Batch, Gftt, GfttParams, GateParams, KltParams, StereoRig, TrackPool, VTError,  # noqa: F401
                 LIB_PATH,
                 header_functions)
