"""GB300-native 3D method-of-characteristics transport sweep.

The compute path lives in ``libmoc3d.so`` (C ABI in ``include/moc.h``):
host C++ for the 2D cyclic tracking, hand-written sm_103a CUDA kernels for
the on-the-fly 3D segment generation, the preloaded/on-the-fly transport
sweep, the source update and the FP64 reductions.  This package is the
ctypes binding (argument marshalling only) plus the build script.
"""
from ._moc import (MOC_FP32, MOC_FP64, MOC_SCHED_ROWS_WITH_SIGMA, MOC_SCHED_TRACKS_NATURAL, MOC_SCHED_UNITS_NATURAL,
                   MOC_TALLY_AUTO, MOC_TALLY_GLOBAL, MOC_TALLY_SHARED,
                   Geometry, MocError, Server, Tracks, autotune, batch_step, load,
                   measure_ex2_rate, measure_unit_rates, eval_attenuation_f64, eval_attenuation_f32, track_params)

__all__ = ["Geometry", "Tracks", "Server", "MocError", "autotune", "batch_step", "load",
           "track_params", "measure_ex2_rate", "measure_unit_rates", "eval_attenuation_f64", "eval_attenuation_f32",
           "MOC_FP32", "MOC_FP64", "MOC_TALLY_AUTO", "MOC_TALLY_SHARED", "MOC_TALLY_GLOBAL",
           "MOC_SCHED_UNITS_NATURAL", "MOC_SCHED_TRACKS_NATURAL", "MOC_SCHED_ROWS_WITH_SIGMA"]
