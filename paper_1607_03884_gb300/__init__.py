"""Batched Radau IIA integration of constant-pressure reactor states on GB300.

The CUDA library (libkin.so, C ABI in include/kin.h) does all the work;
``kin`` is its ctypes binding and ``synth`` the seeded input generator.
"""
from . import synth  # noqa: F401
from .kin import (KinError, Mechanism, radau_constants, lib, options,  # noqa: F401
                  COUNTER_NAMES, LAYOUT_PLAIN, LAYOUT_QUEUE)
