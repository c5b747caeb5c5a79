"""GB300-native hierarchically compressed radiosity view-factor solves.

The compute lives in libvf (CUDA for sm_103a, C ABI in include/vf.h); this
package is its Python binding (``vf``) and build script (``build``).
"""
from .vf import *  # noqa: F401,F403
from .vf import VFError, load  # noqa: F401
