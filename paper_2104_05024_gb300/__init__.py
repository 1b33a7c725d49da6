"""GB300-native kernel-free boundary integral (KFBI) library for the
FitzHugh-Nagumo bidomain equations.  The compute path is the CUDA library
libkfbi.so (include/kfbi.h); ``kfbi`` is its thin ctypes binding."""
from . import kfbi  # noqa: F401
