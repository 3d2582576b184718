"""B300-native QTT / MPS time step for 2-D incompressible Navier-Stokes.

The compute path is the CUDA library libqtt_b300.so (C ABI in
include/qtt.h); :mod:`paper_2406_17823_b300.qtt` is its Python binding.
"""
from .qtt import (PREC_FP64, PREC_MIXED, LEARNED_OFF, LEARNED_LOG, LEARNED_ON,  # noqa: F401
                  RHS_EXPLICIT, RHS_IMPLICIT, PROJ_PENALTY, PROJ_SPECTRAL,
                  MLP_PARAMS, Batch, Context, MPS, Params, QttError, EXPORTS, lib)
