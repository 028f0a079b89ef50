"""FP64 CPU oracle for the MIPWA likelihood (arXiv:1703.03284, Eq. 1, Secs. 2 and 4).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product package never
imports this module, and this module never imports the product package.

The arithmetic lives in ``mipwa_oracle.cpp`` (plain C++, IEEE double,
``std::complex<double>``); this file only compiles it with g++ and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mipwa_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_RES = 8
MAX_KNOTS = 128

OK, EINVAL, ENONPOS = 0, -1, -3
# S-wave knot parametrisations: (a_k, phi_k) or (Re, Im) of the knot values
SWAVE_FORMS = {"magphase": 0, "reim": 1}


class OracleModel(ctypes.Structure):
    """Mirror of ``oracle_model`` in mipwa_oracle.cpp."""

    _fields_ = [
        ("mD", ctypes.c_double),
        ("m1", ctypes.c_double),
        ("m2", ctypes.c_double),
        ("n_res", ctypes.c_int),
        ("mass", ctypes.c_double * MAX_RES),
        ("width", ctypes.c_double * MAX_RES),
        ("spin", ctypes.c_int * MAX_RES),
        ("n_knots", ctypes.c_int),
        ("knots", ctypes.c_double * MAX_KNOTS),
        ("r_res", ctypes.c_double),
        ("r_D", ctypes.c_double),
        ("swave_form", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, no FMA contraction)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            pd = ctypes.POINTER(ctypes.c_double)
            pm = ctypes.POINTER(OracleModel)
            pu8 = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_q.restype = d
            lib.oracle_q.argtypes = [pm, d]
            lib.oracle_p.restype = d
            lib.oracle_p.argtypes = [pm, d]
            lib.oracle_s23_range.argtypes = [pm, d, pd, pd]
            lib.oracle_barrier.restype = d
            lib.oracle_barrier.argtypes = [i32, d, d]
            lib.oracle_zemach.restype = d
            lib.oracle_zemach.argtypes = [pm, i32, d, d]
            lib.oracle_propagator.argtypes = [pm, i32, d, pd, pd]
            lib.oracle_resonance.argtypes = [pm, i32, d, d, pd, pd]
            lib.oracle_spline_second_derivs.argtypes = [i32, pd, pd, pd]
            lib.oracle_spline_eval.argtypes = [i32, pd, pd, pd, i64, pd, pd]
            lib.oracle_inside.argtypes = [pm, i64, pd, pu8, i32]
            lib.oracle_amp.argtypes = [pm, pd, i64, pd, pd, pd]
            lib.oracle_basis.argtypes = [pm, i64, pd, pd]
            lib.oracle_density.argtypes = [pm, pd, i64, pd, pd, i32]
            lib.oracle_nll_grad.argtypes = [pm, pd, i64, pd, i64, pd, pd, pd, i32]
            lib.oracle_nll_grad_w.argtypes = [pm, pd, i64, pd, i64, pd, pd, pd, pd, i32]
            lib.oracle_nll.argtypes = [pm, pd, i64, pd, i64, pd, pd, i32]
            lib.oracle_count_flops.argtypes = [pm, pd, i64, pd, i32, i32, i32, pd]
            lib.oracle_nll_grad_local.argtypes = [pm, pd, i64, pd, i64, pd, pd, pd, pd, i32]
            for f in ("oracle_inside", "oracle_amp", "oracle_basis", "oracle_density",
                      "oracle_nll_grad", "oracle_nll_grad_w", "oracle_nll",
                      "oracle_count_flops", "oracle_nll_grad_local"):
                getattr(lib, f).restype = i32
            _lib = lib
    return _lib


def _pd(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _events(x) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("events must have shape (n, 2): columns s12, s13")
    return a


def default_threads() -> int:
    return os.cpu_count() or 1


def make_model(model) -> OracleModel:
    """Build the ctypes model from any object with the attributes of
    ``synth.ModelSpec`` (mD, m1, m2, resonances[(mass, width, spin)], knots,
    r_res, r_D, and optionally swave_form: "magphase" (default) or "reim")."""
    m = OracleModel()
    m.mD, m.m1, m.m2 = float(model.mD), float(model.m1), float(model.m2)
    res = list(model.resonances)
    if len(res) > MAX_RES:
        raise ValueError("too many resonances for the oracle")
    m.n_res = len(res)
    for r, (mass, width, spin) in enumerate(res):
        m.mass[r], m.width[r], m.spin[r] = float(mass), float(width), int(spin)
    knots = np.asarray(model.knots, dtype=np.float64)
    if len(knots) > MAX_KNOTS:
        raise ValueError("too many knots for the oracle")
    m.n_knots = len(knots)
    for k, x in enumerate(knots):
        m.knots[k] = float(x)
    m.r_res, m.r_D = float(model.r_res), float(model.r_D)
    form = getattr(model, "swave_form", "magphase")
    if form not in SWAVE_FORMS:
        raise ValueError(f"unknown S-wave form {form!r}")
    m.swave_form = SWAVE_FORMS[form]
    return m


class Oracle:
    """Callable handle on the FP64 oracle for one decay model."""

    def __init__(self, model):
        self.spec = model
        self.m = make_model(model)
        self.lib = _load()
        self.n_params = 2 * self.m.n_res + 2 * self.m.n_knots

    def _params(self, params) -> np.ndarray:
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        if p.shape != (self.n_params,):
            raise ValueError(f"expected {self.n_params} parameters, got {p.shape}")
        return p

    # -- pieces --
    def q(self, s):
        return self.lib.oracle_q(ctypes.byref(self.m), float(s))

    def p(self, s):
        return self.lib.oracle_p(ctypes.byref(self.m), float(s))

    def s23_range(self, s12):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        self.lib.oracle_s23_range(ctypes.byref(self.m), float(s12), ctypes.byref(lo),
                                  ctypes.byref(hi))
        return lo.value, hi.value

    def zemach(self, L, s, s_other):
        return self.lib.oracle_zemach(ctypes.byref(self.m), int(L), float(s), float(s_other))

    def propagator(self, r, s):
        re, im = ctypes.c_double(), ctypes.c_double()
        self.lib.oracle_propagator(ctypes.byref(self.m), int(r), float(s), ctypes.byref(re),
                                   ctypes.byref(im))
        return complex(re.value, im.value)

    def resonance(self, r, s, s_other):
        re, im = ctypes.c_double(), ctypes.c_double()
        self.lib.oracle_resonance(ctypes.byref(self.m), int(r), float(s), float(s_other),
                                  ctypes.byref(re), ctypes.byref(im))
        return complex(re.value, im.value)

    # -- vectorised --
    def inside(self, events, threads: int | None = None) -> np.ndarray:
        ev = _events(events)
        out = np.zeros(len(ev), dtype=np.uint8)
        self.lib.oracle_inside(ctypes.byref(self.m), len(ev), _pd(ev),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                               threads or default_threads())
        return out.astype(bool)

    def amp(self, params, events) -> np.ndarray:
        p, ev = self._params(params), _events(events)
        re, im = np.empty(len(ev)), np.empty(len(ev))
        rc = self.lib.oracle_amp(ctypes.byref(self.m), _pd(p), len(ev), _pd(ev), _pd(re), _pd(im))
        if rc != OK:
            raise ValueError(f"oracle_amp failed ({rc})")
        return re + 1j * im

    def basis(self, events) -> np.ndarray:
        ev = _events(events)
        out = np.empty((len(ev), self.m.n_res, 2))
        rc = self.lib.oracle_basis(ctypes.byref(self.m), len(ev), _pd(ev), _pd(out))
        if rc != OK:
            raise ValueError(f"oracle_basis failed ({rc})")
        return out[..., 0] + 1j * out[..., 1]

    def density(self, params, events, threads: int | None = None) -> np.ndarray:
        p, ev = self._params(params), _events(events)
        out = np.empty(len(ev))
        rc = self.lib.oracle_density(ctypes.byref(self.m), _pd(p), len(ev), _pd(ev), _pd(out),
                                     threads or default_threads())
        if rc != OK:
            raise ValueError(f"oracle_density failed ({rc})")
        return out

    def amp2(self, params, events) -> np.ndarray:
        return np.abs(self.amp(params, events)) ** 2

    def nll(self, params, data, norm, threads: int | None = None, norm_weights=None) -> float:
        v, _ = self._nll_grad(params, data, norm, False, threads, norm_weights)
        return v

    def nll_grad(self, params, data, norm, threads: int | None = None, norm_weights=None):
        """-2 ln L and its gradient; norm_weights (one per normalisation point,
        None: all 1) make the normalisation integral a weighted mean."""
        return self._nll_grad(params, data, norm, True, threads, norm_weights)

    def _nll_grad(self, params, data, norm, want_grad, threads, norm_weights=None):
        p = self._params(params)
        d = _events(data) if len(data) else np.zeros((0, 2))
        n = _events(norm)
        w = None
        if norm_weights is not None:
            w = np.ascontiguousarray(norm_weights, dtype=np.float64)
            if w.shape != (len(n),):
                raise ValueError("one weight per normalisation point")
        out = ctypes.c_double()
        g = np.empty(self.n_params) if want_grad else None
        rc = self.lib.oracle_nll_grad_w(ctypes.byref(self.m), _pd(p), len(d), _pd(d), len(n),
                                        _pd(n), _pd(w) if w is not None else None,
                                        ctypes.byref(out), _pd(g) if want_grad else None,
                                        threads or default_threads())
        if rc != OK:
            raise ArithmeticError(f"oracle_nll_grad failed ({rc})")
        return out.value, g


    def nll_grad_local(self, params, data, norm, threads: int | None = None,
                       norm_weights=None):
        """-2 ln L and its gradient with the spline part of the gradient summed
        in the local (segment-bin) form and mapped to the knots once."""
        p = self._params(params)
        d = _events(data) if len(data) else np.zeros((0, 2))
        n = _events(norm)
        w = None if norm_weights is None else np.ascontiguousarray(norm_weights, dtype=np.float64)
        out = ctypes.c_double()
        g = np.empty(self.n_params)
        rc = self.lib.oracle_nll_grad_local(ctypes.byref(self.m), _pd(p), len(d), _pd(d), len(n),
                                            _pd(n), _pd(w) if w is not None else None,
                                            ctypes.byref(out), _pd(g),
                                            threads or default_threads())
        if rc != OK:
            raise ArithmeticError(f"oracle_nll_grad_local failed ({rc})")
        return out.value, g

    def count_flops(self, params, events, is_data: bool, grad: bool, cached: bool = False) -> dict:
        """Mean event-dependent operations per event of one evaluation (see
        oracle_count_flops): adds, muls, divs, sqrts, funcs and their total."""
        p, ev = self._params(params), _events(events)
        out = np.zeros(6)
        rc = self.lib.oracle_count_flops(ctypes.byref(self.m), _pd(p), len(ev), _pd(ev),
                                         int(is_data), int(grad), int(cached), _pd(out))
        if rc != OK:
            raise ValueError(f"oracle_count_flops failed ({rc})")
        return dict(zip(("add", "mul", "div", "sqrt", "func", "total"), out.tolist()))


def spline_second_derivs(x, y) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    M = np.empty_like(x)
    lib.oracle_spline_second_derivs(len(x), _pd(x), _pd(y), _pd(M))
    return M


def spline_eval(x, y, M, s) -> np.ndarray:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    s = np.ascontiguousarray(np.atleast_1d(s), dtype=np.float64)
    out = np.empty_like(s)
    lib.oracle_spline_eval(len(x), _pd(x), _pd(y), _pd(M), len(s), _pd(s), _pd(out))
    return out


def barrier(L, z, z0) -> float:
    return _load().oracle_barrier(int(L), float(z), float(z0))
