"""GB300-native time-domain Casimir-force library (arXiv:0906.5170).

The computation lives in libcasimir.so (include/casimir.h): a host planner and
hand-written CUDA kernels for sm_103a.  This package only builds and binds it.
"""
from .capi import (  # noqa: F401
    Context, Plan, Ticket, CasimirError, lib, header_functions, MarshalledProblem,
)
