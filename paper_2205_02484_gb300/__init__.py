"""GB300-native GR-MHD conservative step (the hot path of cuHARM, arXiv 2205.02484).

The compute lives in ``libgrmhd.so`` (CUDA for sm_103a, C ABI in
``include/grmhd.h``); ``grmhd`` is its thin Python binding.
"""
from . import grmhd  # noqa: F401
from .grmhd import (  # noqa: F401
    init_grid, set_metric, init_torus, set_state, get_state, step, sync, diagnostics,
    con2prim, prim2cons, fluxes, default_grid, default_phys, GrmhdError,
)
