"""GB300 (sm_103a) library for the space-time boundary-regularised boundary integral method of
Klaseboer, Sepehrirahnama & Chan (arXiv 1706.07919).

The computation lives in libbie.so (C ABI: include/bie.h); `binding` marshals arguments to it and
`Solver` bundles a context with torch-allocated outputs.  Nothing here computes on the host.
"""
from __future__ import annotations

from .solver import Solver  # noqa: F401
