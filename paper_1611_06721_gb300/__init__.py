"""GB300-native (sm_103a) hot path of the semi-explicit eddy-current scheme
with multiple right-hand side start vectors (SPE and POD).

The compute lives in ``_lib/libmqs.so`` (hand-written CUDA, C ABI in
``include/mqs.h``); :mod:`.binding` marshals arguments to it.
"""
from .binding import (  # noqa: F401
    DEBUG, EXPORTS, LIB_PATH, START_CSPE, START_POD, START_PREV, START_SPE, START_ZERO, Batch, MqsError, Solver,
    SolverOptions, debug_check, eddy_loss, load,
)
