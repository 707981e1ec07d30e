"""GB300-native SNMPBB: nonmonotone projected Barzilai-Borwein symmetric NMF.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
include/snmf.h); :mod:`.snmf` is its ctypes binding.  Importing the package does
not load the library; the first binding call does, and fails loudly if it has not
been built.
"""
from . import snmf  # noqa: F401

__all__ = ["snmf"]
