"""GB300-native ensemble electron Monte Carlo for wurtzite GaN (Hao et al.,
arXiv:1707.09073): the flight/scatter/tally hot path as sm_103a CUDA kernels
behind the C ABI of include/emc.h, with a thin ctypes binding."""
from .emc import (Context, EmcConfig, EmcError, FP32, FP64, GEOM_BULK, GEOM_NANOWIRE, TALLY_CHARGE,
                  TALLY_CROSSINGS, TALLY_EVENTS, TALLY_EVENTS_CELL, TALLY_FIELD, TALLY_HEAT, TALLY_HEAT_J, TALLY_OBS, TALLY_PHI,
                  lib, make_config)

__all__ = ["Context", "EmcConfig", "EmcError", "FP32", "FP64", "GEOM_BULK", "GEOM_NANOWIRE", "TALLY_CHARGE",
           "TALLY_CROSSINGS", "TALLY_EVENTS", "TALLY_EVENTS_CELL", "TALLY_FIELD", "TALLY_HEAT", "TALLY_HEAT_J", "TALLY_OBS",
           "TALLY_PHI", "lib", "make_config"]
