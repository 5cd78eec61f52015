"""GB300 (sm_103a) implementation of RLFC random-access light-field decode and
rendering (Pratapa & Manocha, I3D 2019).  The compute path is librlfc.so (C ABI
in include/rlfc.h); this package builds it (build) and binds it (rlfc)."""
from .buildlib import LIB, build  # noqa: F401
from . import rlfc  # noqa: F401

__all__ = ["build", "LIB", "rlfc"]
