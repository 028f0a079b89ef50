"""Python binding of the MIPWA likelihood engine: one class whose methods carry
the names of the C entry points (include/mipwa.h) and only marshal arguments.

Events may be numpy arrays or torch tensors of shape (n, 2) holding (s12, s13)
in float64 or float32; CUDA tensors are passed to the library as device
pointers, everything else as host pointers.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

from . import _lib
from ._lib import F32, F64


def _config_dict(cfg) -> dict:
    return {"norm_chunk": cfg.norm_chunk, "data_chunk": cfg.data_chunk, "block": cfg.block,
            "blocks_per_sm": cfg.blocks_per_sm}


class MipwaError(RuntimeError):
    def __init__(self, status: int, message: str, n_outside: int = 0):
        self.status = status
        self.n_outside = n_outside
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {message}")


def _torch():
    import torch
    return torch


def _event_buffer(x):
    """Return (pointer, n, dtype code, on_device, keepalive) for an (n, 2) array."""
    try:
        torch = _torch()
        is_tensor = isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover - torch is part of the runtime
        is_tensor = False
    if is_tensor:
        if x.dim() != 2 or x.shape[1] != 2:
            raise ValueError("events must have shape (n, 2)")
        if x.dtype not in (torch.float32, torch.float64):
            raise ValueError("events must be float32 or float64")
        t = x.contiguous()
        code = F32 if t.dtype == torch.float32 else F64
        return t.data_ptr(), t.shape[0], code, int(t.is_cuda), t
    a = np.asarray(x)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("events must have shape (n, 2)")
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    a = np.ascontiguousarray(a)
    code = F32 if a.dtype == np.float32 else F64
    return a.ctypes.data, a.shape[0], code, 0, a


class Likelihood:
    """One library context (``mipwa_ctx``) on one CUDA device."""

    def __init__(self, device: int = 0, compute_mode: int = F64):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        rc = self._lib.mipwa_create(ctypes.byref(h), int(device), int(compute_mode))
        if rc != _lib.OK:
            raise MipwaError(rc, f"mipwa_create(device={device}) failed")
        self._h = h
        self.device = device
        self.n_params = -1
        self.follow_torch_stream = True
        self._stream = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.mipwa_destroy(h)
            self._h = None

    def _follow_stream(self):
        """Queue the library's work on torch's current stream of this device, so
        that it is ordered with the torch work that made or reads its tensors."""
        torch = _torch()
        if self.follow_torch_stream and torch.cuda.is_available():
            s = torch.cuda.current_stream(self.device).cuda_stream
            if s != self._stream:
                self._check(self._lib.mipwa_set_stream(self._h, ctypes.c_void_p(s)))
                self._stream = s

    def _check(self, rc: int, n_outside: int = 0):
        if rc != _lib.OK:
            raise MipwaError(rc, self.last_error(), n_outside)

    # ---------------------------------------------------------------- setup
    def set_stream(self, stream):
        """Queue work on a torch.cuda.Stream or raw cudaStream_t handle and stop
        following torch's current stream."""
        ptr = getattr(stream, "cuda_stream", stream)
        self.follow_torch_stream = False
        self._check(self._lib.mipwa_set_stream(self._h, ctypes.c_void_p(ptr)))
        self._stream = ptr

    def set_compute_mode(self, mode: int):
        self._check(self._lib.mipwa_set_compute_mode(self._h, int(mode)))

    def set_masses(self, mD: float, m1: float, m2: float):
        self._check(self._lib.mipwa_set_masses(self._h, mD, m1, m2))

    def set_model(self, resonances: Sequence, knots: Sequence[float], r_res: float, r_D: float):
        res = (_lib.Resonance * max(len(resonances), 1))()
        for i, (mass, width, spin) in enumerate(resonances):
            res[i] = _lib.Resonance(float(mass), float(width), int(spin))
        kn = np.ascontiguousarray(knots, dtype=np.float64)
        self._check(self._lib.mipwa_set_model(
            self._h, res, len(resonances), kn.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            len(kn), float(r_res), float(r_D)))
        self.n_params = self.num_params()
        self.n_res = len(resonances)

    def set_spec(self, spec):
        """set_masses + set_model (+ set_swave_form) from an object with mD, m1,
        m2, resonances, knots, r_res, r_D (and optionally swave_form)
        attributes."""
        self.set_masses(spec.mD, spec.m1, spec.m2)
        self.set_model(spec.resonances, spec.knots, spec.r_res, spec.r_D)
        self.set_swave_form(getattr(spec, "swave_form", "magphase"))

    def set_swave_form(self, form):
        """"magphase" (knot block [a_k, phi_k]) or "reim" (knot block [x_k, y_k],
        A0 = x(s) + i y(s)); or the MIPWA_SWAVE_* code."""
        code = {"magphase": _lib.SWAVE_MAGPHASE, "reim": _lib.SWAVE_REIM}.get(form, form)
        self._check(self._lib.mipwa_set_swave_form(self._h, int(code)))

    def enable_norm_gram(self, on: bool = True):
        """Normalisation from per-cell moments of the normalisation sample
        (Re/Im form only)."""
        self._check(self._lib.mipwa_enable_norm_gram(self._h, int(bool(on))))

    def build_norm_gram(self):
        self._follow_stream()
        self._check(self._lib.mipwa_build_norm_gram(self._h))

    def set_resonances(self, resonances: Sequence):
        """New (mass, width, spin) for the model's resonances (same count);
        knots, radii and stored samples are kept."""
        res = (_lib.Resonance * max(len(resonances), 1))()
        for i, (mass, width, spin) in enumerate(resonances):
            res[i] = _lib.Resonance(float(mass), float(width), int(spin))
        self._check(self._lib.mipwa_set_resonances(self._h, res, len(resonances)))

    def _set(self, fn, x):
        self._follow_stream()
        ptr, n, code, on_dev, keep = _event_buffer(x)
        n_out = ctypes.c_int64(0)
        rc = fn(self._h, ctypes.c_void_p(ptr), n, code, on_dev, ctypes.byref(n_out))
        del keep
        self._check(rc, n_out.value)

    def set_events(self, x):
        self._set(self._lib.mipwa_set_events, x)

    def set_norm_sample(self, x, weights=None):
        """Normalisation points (n, 2); optional weights (n,), one per point,
        make the normalisation integral their weighted mean. The weights are
        converted to the points' dtype and must live where the points do."""
        if weights is None:
            self._set(self._lib.mipwa_set_norm_sample, x)
            return
        self._follow_stream()
        ptr, n, code, on_dev, keep = _event_buffer(x)
        torch = _torch()
        if on_dev:
            w = torch.as_tensor(weights, device=keep.device)
            w = w.to(keep.dtype).contiguous()
            wptr = w.data_ptr()
        else:
            w = np.ascontiguousarray(weights, dtype=np.float32 if code == F32 else np.float64)
            wptr = w.ctypes.data
        if w.shape != (n,):
            raise ValueError("one weight per normalisation point")
        n_out = ctypes.c_int64(0)
        rc = self._lib.mipwa_set_norm_sample_weighted(self._h, ctypes.c_void_p(ptr),
                                                      ctypes.c_void_p(wptr), n, code, on_dev,
                                                      ctypes.byref(n_out))
        del keep, w
        self._check(rc, n_out.value)

    def enable_basis_cache(self, on: bool = True):
        self._check(self._lib.mipwa_enable_basis_cache(self._h, int(bool(on))))

    def set_toys(self, events, offsets):
        """Toy data samples back to back; toy t owns events[offsets[t]:offsets[t+1]]."""
        self._follow_stream()
        ptr, n, code, on_dev, keep = _event_buffer(events)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        n_out = ctypes.c_int64(0)
        rc = self._lib.mipwa_set_toys(self._h, ctypes.c_void_p(ptr), n, code, on_dev,
                                      off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      len(off) - 1, ctypes.byref(n_out))
        del keep
        self._check(rc, n_out.value)
        self.n_toys = len(off) - 1

    def nll_grad_toys(self, params):
        """params: (n_toys, P) -> (nll (n_toys,), grad (n_toys, P))."""
        self._follow_stream()
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        if p.shape != (self.n_toys, self.n_params):
            raise ValueError(f"expected params of shape {(self.n_toys, self.n_params)}")
        nll = np.empty(self.n_toys)
        g = np.empty_like(p)
        pd = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.mipwa_nll_grad_toys(self._h, p.ctypes.data_as(pd),
                                                  nll.ctypes.data_as(pd), g.ctypes.data_as(pd)))
        return nll, g

    def nll_toys(self, params):
        """params: (n_toys, P) -> nll (n_toys,), without the gradient."""
        self._follow_stream()
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        if p.shape != (self.n_toys, self.n_params):
            raise ValueError(f"expected params of shape {(self.n_toys, self.n_params)}")
        nll = np.empty(self.n_toys)
        pd = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.mipwa_nll_toys(self._h, p.ctypes.data_as(pd),
                                             nll.ctypes.data_as(pd)))
        return nll

    def toys_autotune(self, params) -> dict:
        """Time the batched evaluation over its launch configurations, keep the
        fastest; returns it as a dict with "n_timed" (0: a cached choice)."""
        self._follow_stream()
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        cfg = _lib.ToysConfig()
        n_timed = ctypes.c_int(0)
        self._check(self._lib.mipwa_toys_autotune(
            self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cfg),
            ctypes.byref(n_timed)))
        out = _config_dict(cfg)
        out["n_timed"] = n_timed.value
        return out

    def toys_norm_tc(self, params, mode: int = 0):
        """mipwa_toys_norm_tc: (integrals per toy, kernel ms) for mode 0, or
        (the spline products [4, 128, 64] of the first tile, kernel ms) for
        mode 1."""
        self._follow_stream()
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
        if p.shape != (self.n_toys, self.n_params):
            raise ValueError(f"expected params of shape {(self.n_toys, self.n_params)}")
        out = np.zeros(self.n_toys if mode == 0 else 4 * 128 * 64)
        ms = ctypes.c_double(0.0)
        pd = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.mipwa_toys_norm_tc(self._h, p.ctypes.data_as(pd), int(mode),
                                                 out.ctypes.data_as(pd), ctypes.byref(ms)))
        return (out if mode == 0 else out.reshape(4, 128, 64)), ms.value

    def set_toys_graph(self, on: bool = True):
        self._check(self._lib.mipwa_set_toys_graph(self._h, int(bool(on))))

    def set_toys_config(self, norm_chunk: int = 0, data_chunk: int = 0, block: int = 0,
                        blocks_per_sm: int = 0):
        """Launch configuration of the batched evaluation (0 keeps a chunk or
        the block size; blocks_per_sm 0 = as many as fit)."""
        cfg = _lib.ToysConfig(int(norm_chunk), int(data_chunk), int(block), int(blocks_per_sm))
        self._check(self._lib.mipwa_set_toys_config(self._h, ctypes.byref(cfg)))

    def toys_config(self) -> dict:
        cfg = _lib.ToysConfig()
        self._check(self._lib.mipwa_get_toys_config(self._h, ctypes.byref(cfg)))
        return _config_dict(cfg)

    def set_toys_tune_file(self, path):
        """File of autotuner choices (looked up, then appended to); None: off."""
        arg = None if path is None else os.fsencode(path)
        self._check(self._lib.mipwa_set_toys_tune_file(self._h, arg))

    def num_params(self) -> int:
        return int(self._lib.mipwa_num_params(self._h))

    # -------------------------------------------------------------- compute
    def _params(self, params) -> np.ndarray:
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))
        if p.shape[0] != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.shape[0]}")
        return p

    def nll(self, params) -> float:
        self._follow_stream()
        p = self._params(params)
        out = ctypes.c_double()
        self._check(self._lib.mipwa_nll(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(out)))
        return out.value

    def nll_grad(self, params):
        self._follow_stream()
        p = self._params(params)
        out = ctypes.c_double()
        g = np.empty_like(p)
        self._check(self._lib.mipwa_nll_grad(
            self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(out),
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out.value, g

    def nll_grad_streamed(self, params, data, norm):
        """Set both samples from HOST arrays (n, 2) of one dtype (pinned
        tensors copy fastest) and evaluate -2 ln L and its gradient in one
        pipelined call (mipwa_nll_grad_streamed)."""
        self._follow_stream()
        p = self._params(params)
        dptr, nd, code_d, on_d, kd = _event_buffer(data)
        nptr, nn, code_n, on_n, kn = _event_buffer(norm)
        if on_d or on_n:
            raise ValueError("nll_grad_streamed takes host arrays")
        if nd > 0 and code_d != code_n:
            raise ValueError("data and normalisation samples must share a dtype")
        out = ctypes.c_double()
        g = np.empty_like(p)
        n_out = ctypes.c_int64(0)
        pd = ctypes.POINTER(ctypes.c_double)
        rc = self._lib.mipwa_nll_grad_streamed(
            self._h, p.ctypes.data_as(pd), ctypes.c_void_p(dptr), nd, ctypes.c_void_p(nptr), nn,
            code_n, ctypes.byref(out), g.ctypes.data_as(pd), ctypes.byref(n_out))
        del kd, kn
        self._check(rc, n_out.value)
        return out.value, g

    def nll_grad_bw(self, params):
        """(NLL, dNLL/dparams, [dNLL/dm_r, dNLL/dGamma_r]_r) in FP64 at the
        current resonance masses and widths."""
        self._follow_stream()
        p = self._params(params)
        pd = ctypes.POINTER(ctypes.c_double)
        out = ctypes.c_double()
        g = np.empty_like(p)
        gbw = np.empty(2 * self.n_res)
        self._check(self._lib.mipwa_nll_grad_bw(self._h, p.ctypes.data_as(pd), ctypes.byref(out),
                                                g.ctypes.data_as(pd), gbw.ctypes.data_as(pd)))
        return out.value, g, gbw

    def amp2(self, params, events):
        """|A|^2 per event (0 outside the Dalitz plot) for a CUDA tensor of events;
        returns a float64 CUDA tensor."""
        torch = _torch()
        if not (isinstance(events, torch.Tensor) and events.is_cuda):
            raise ValueError("amp2 takes a CUDA tensor of events")
        self._follow_stream()
        ptr, n, code, _, keep = _event_buffer(events)
        out = torch.empty(n, dtype=torch.float64, device=events.device)
        p = self._params(params)
        self._check(self._lib.mipwa_amp2(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.c_void_p(ptr), n, code,
                                         ctypes.c_void_p(out.data_ptr())))
        del keep
        return out

    def inside(self, events):
        """Boolean CUDA tensor: event inside the Dalitz plot."""
        torch = _torch()
        if not (isinstance(events, torch.Tensor) and events.is_cuda):
            raise ValueError("inside takes a CUDA tensor of events")
        self._follow_stream()
        ptr, n, code, _, keep = _event_buffer(events)
        out = torch.empty(n, dtype=torch.uint8, device=events.device)
        self._check(self._lib.mipwa_inside(self._h, ctypes.c_void_p(ptr), n, code,
                                           ctypes.c_void_p(out.data_ptr())))
        del keep
        return out.bool()

    def stored_sample(self, which: str = "data"):
        """The stored data ("data") or normalisation ("norm") sample as an
        (n, 2) CUDA tensor in the order the library holds it: grouped by
        spline cell once a model is set (stable within a cell)."""
        torch = _torch()
        code = {"data": _lib.SAMPLE_DATA, "norm": _lib.SAMPLE_NORM}[which]
        n, dt = ctypes.c_int64(0), ctypes.c_int(0)
        self._check(self._lib.mipwa_get_sample(self._h, code, None, 0, ctypes.byref(n),
                                               ctypes.byref(dt)))
        dtype = torch.float32 if dt.value == _lib.F32 else torch.float64
        out = torch.empty((n.value, 2), dtype=dtype, device=f"cuda:{self.device}")
        self._follow_stream()
        self._check(self._lib.mipwa_get_sample(self._h, code, ctypes.c_void_p(out.data_ptr()),
                                               n.value, None, None))
        return out

    # ----------------------------------------------------------- diagnostics
    def set_timing(self, on: bool = True):
        self._check(self._lib.mipwa_set_timing(self._h, int(bool(on))))

    def kernel_time(self):
        """(summed milliseconds, launches) of the fused event kernel since timing was on."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._lib.mipwa_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def last_error(self) -> str:
        s = self._lib.mipwa_last_error(self._h)
        return s.decode() if s else ""

    def launch_count(self) -> int:
        return int(self._lib.mipwa_launch_count(self._h))


PROBES = {"ffma": _lib.PROBE_FFMA, "ffma2": _lib.PROBE_FFMA2, "dfma": _lib.PROBE_DFMA,
          "mufu": _lib.PROBE_MUFU}


def probe_peak(kind: str, device: int = 0, target_ms: float = 100.0) -> tuple[float, float]:
    """mipwa_probe_peak: (operations per second, timed milliseconds) of one
    pipe ("ffma", "ffma2", "dfma" in flops/s; "mufu" in approximations/s)."""
    lib = _lib.load()
    ops = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    rc = lib.mipwa_probe_peak(int(device), PROBES[kind], float(target_ms), ctypes.byref(ops),
                              ctypes.byref(ms))
    if rc != _lib.OK:
        raise MipwaError(rc, f"mipwa_probe_peak({kind}) failed")
    return ops.value, ms.value


def nll_grad_noalloc(spec, params, data, norm, compute_mode: int = F64):
    """mipwa_nll_grad_noalloc through the C ABI: no context and no device
    allocation inside the library. `data` and `norm` are CUDA tensors (n, 2) of
    one dtype on one device, which is the device the call runs on; returns
    (NLL, gradient) read back from a caller-owned buffer."""
    import torch
    lib = _lib.load()
    if not (isinstance(data, torch.Tensor) and data.is_cuda and isinstance(norm, torch.Tensor)
            and norm.is_cuda and data.dtype == norm.dtype):
        raise ValueError("data and norm must be CUDA tensors of one dtype")
    if data.device != norm.device:
        raise ValueError("data and norm must be on the same device")
    device = data.device.index if data.device.index is not None else torch.cuda.current_device()
    d_ptr, nd, code, _, kd = _event_buffer(data)
    n_ptr, nn, code_n, _, kn = _event_buffer(norm)
    res = (_lib.Resonance * max(len(spec.resonances), 1))()
    for i, (mass, width, spin) in enumerate(spec.resonances):
        res[i] = _lib.Resonance(float(mass), float(width), int(spin))
    knots = np.ascontiguousarray(spec.knots, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    P = 2 * len(spec.resonances) + 2 * len(knots)
    if p.shape != (P,):
        raise ValueError(f"expected {P} parameters")
    out = torch.empty(1 + P, dtype=torch.float64, device=data.device)
    stream = torch.cuda.current_stream(data.device).cuda_stream
    pd = ctypes.POINTER(ctypes.c_double)
    rc = lib.mipwa_nll_grad_noalloc(
        int(device), int(compute_mode), float(spec.mD), float(spec.m1), float(spec.m2), res,
        len(spec.resonances), knots.ctypes.data_as(pd), len(knots), float(spec.r_res),
        float(spec.r_D), ctypes.c_void_p(d_ptr), nd, ctypes.c_void_p(n_ptr), nn, code,
        p.ctypes.data_as(pd), ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    del kd, kn
    if rc != _lib.OK:
        raise MipwaError(rc, "mipwa_nll_grad_noalloc failed")
    o = out.cpu().numpy()
    return float(o[0]), o[1:].copy()

