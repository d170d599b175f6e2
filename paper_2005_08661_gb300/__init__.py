"""GB300-native regularised 3-D field-map estimation (Lin & Fessler, arXiv 2005.08661).

The estimator (IC(0)-preconditioned Polak-Ribiere NCG with the monotonic line search
on the phase-wrapping cost of Eq. 5) runs in hand-written sm_103a CUDA kernels behind
the C ABI of include/fm.h; :class:`FieldMap` is a thin ctypes binding of that ABI.
"""
from .fm import (FieldMap, FieldMapBatch, FmError, FmOpts, load_library, lib_path, EXPORTS, FM_OK, FM_ERR_ARG,
                 FM_ERR_STATE, FM_ERR_CUDA, FM_ERR_NOT_PD, FM_ERR_TIMEOUT, FM_ERR_NONFINITE, FM_ERR_OOM,
                 FM_ERR_SIZE, FM_ERR_FILL)
from .autograd import field_map_cost, field_map_solve

__all__ = ["FieldMap", "FieldMapBatch", "FmError", "FmOpts", "load_library", "lib_path", "EXPORTS", "FM_OK", "FM_ERR_ARG",
           "FM_ERR_STATE", "FM_ERR_CUDA", "FM_ERR_NOT_PD", "FM_ERR_TIMEOUT", "FM_ERR_NONFINITE", "FM_ERR_OOM",
           "FM_ERR_SIZE", "FM_ERR_FILL", "field_map_cost", "field_map_solve"]
