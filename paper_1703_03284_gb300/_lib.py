"""ctypes declarations of ``libmipwa.so`` (the C ABI in include/mipwa.h).

The library is loaded from this package directory. There is no fallback: if
it has not been built, importing the binding raises immediately.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmipwa.so")

OK, EINVAL, EOUTSIDE, ENONPOS, ECUDA, ETIMEOUT, ESTATE, ENOMEM = 0, -1, -2, -3, -4, -5, -6, -7
F64, F32 = 0, 1
SWAVE_MAGPHASE, SWAVE_REIM = 0, 1
SAMPLE_DATA, SAMPLE_NORM = 0, 1
MAX_RES = 4
MAX_KNOTS = 64
MAX_TOYS = 4096
PROBE_FFMA, PROBE_FFMA2, PROBE_DFMA, PROBE_MUFU = 0, 1, 2, 3

STATUS_NAMES = {OK: "MIPWA_OK", EINVAL: "MIPWA_EINVAL", EOUTSIDE: "MIPWA_EOUTSIDE",
                ENONPOS: "MIPWA_ENONPOS", ECUDA: "MIPWA_ECUDA", ETIMEOUT: "MIPWA_ETIMEOUT",
                ESTATE: "MIPWA_ESTATE", ENOMEM: "MIPWA_ENOMEM"}


class Resonance(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("width", ctypes.c_double), ("spin", ctypes.c_int)]


class ToysConfig(ctypes.Structure):
    """Mirror of ``mipwa_toys_config``."""
    _fields_ = [("norm_chunk", ctypes.c_int64), ("data_chunk", ctypes.c_int64),
                ("block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int)]


# (name, restype, argtypes) of every exported function
_vp, _i, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("mipwa_create", _i, [ctypes.POINTER(_vp), _i, _i]),
    ("mipwa_destroy", None, [_vp]),
    ("mipwa_set_stream", _i, [_vp, _vp]),
    ("mipwa_set_compute_mode", _i, [_vp, _i]),
    ("mipwa_set_masses", _i, [_vp, _d, _d, _d]),
    ("mipwa_set_model", _i, [_vp, ctypes.POINTER(Resonance), _i, _pd, _i, _d, _d]),
    ("mipwa_set_resonances", _i, [_vp, ctypes.POINTER(Resonance), _i]),
    ("mipwa_nll_grad_bw", _i, [_vp, _pd, _pd, _pd, _pd]),
    ("mipwa_set_events", _i, [_vp, _vp, _i64, _i, _i, _pi64]),
    ("mipwa_set_norm_sample", _i, [_vp, _vp, _i64, _i, _i, _pi64]),
    ("mipwa_enable_basis_cache", _i, [_vp, _i]),
    ("mipwa_set_swave_form", _i, [_vp, _i]),
    ("mipwa_enable_norm_gram", _i, [_vp, _i]),
    ("mipwa_build_norm_gram", _i, [_vp]),
    ("mipwa_num_params", _i, [_vp]),
    ("mipwa_nll", _i, [_vp, _pd, _pd]),
    ("mipwa_nll_grad", _i, [_vp, _pd, _pd, _pd]),
    ("mipwa_nll_grad_streamed", _i, [_vp, _pd, _vp, _i64, _vp, _i64, _i, _pd, _pd, _pi64]),
    ("mipwa_set_toys", _i, [_vp, _vp, _i64, _i, _i, _pi64, _i, _pi64]),
    ("mipwa_nll_grad_toys", _i, [_vp, _pd, _pd, _pd]),
    ("mipwa_nll_toys", _i, [_vp, _pd, _pd]),
    ("mipwa_toys_autotune", _i, [_vp, _pd, ctypes.POINTER(ToysConfig), ctypes.POINTER(_i)]),
    ("mipwa_set_toys_graph", _i, [_vp, _i]),
    ("mipwa_toys_norm_tc", _i, [_vp, _pd, _i, _pd, _pd]),
    ("mipwa_set_toys_config", _i, [_vp, ctypes.POINTER(ToysConfig)]),
    ("mipwa_get_toys_config", _i, [_vp, ctypes.POINTER(ToysConfig)]),
    ("mipwa_set_toys_tune_file", _i, [_vp, ctypes.c_char_p]),
    ("mipwa_probe_peak", _i, [_i, _i, _d, _pd, _pd]),
    ("mipwa_amp2", _i, [_vp, _pd, _vp, _i64, _i, _vp]),
    ("mipwa_inside", _i, [_vp, _vp, _i64, _i, _vp]),
    ("mipwa_get_sample", _i, [_vp, _i, _vp, _i64, _pi64, ctypes.POINTER(_i)]),
    ("mipwa_set_norm_sample_weighted", _i, [_vp, _vp, _vp, _i64, _i, _i, _pi64]),
    ("mipwa_nll_grad_noalloc", _i, [_i, _i, _d, _d, _d, ctypes.POINTER(Resonance), _i, _pd, _i,
                                    _d, _d, _vp, _i64, _vp, _i64, _i, _pd, _vp, _vp]),
    ("mipwa_set_timing", _i, [_vp, _i]),
    ("mipwa_kernel_time", _i, [_vp, _pd, _pi64]),
    ("mipwa_last_error", ctypes.c_char_p, [_vp]),
    ("mipwa_launch_count", _i64, [_vp]),
]

_lib = None


def load() -> ctypes.CDLL:
    """Load libmipwa.so and declare its functions; raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`"
                " (the CUDA library is required: there is no CPU path)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
