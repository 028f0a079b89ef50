"""Host quasi-Newton minimiser of -2 ln L (the unbinned maximum-likelihood fit
of arXiv:1703.03284, Sec. 2), calling the library's NLL+gradient each step.

Fixed parameters (by default Re c_0, Im c_0: the reference wave) are held at
their start values. Uncertainties come from the Hessian of -2 ln L, built by
central differences of the analytic gradient: cov = 2 H^{-1}.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Sequence

import numpy as np


@dataclasses.dataclass
class FitResult:
    params: np.ndarray
    nll: float
    errors: np.ndarray | None
    n_calls: int
    converged: bool
    message: str
    seconds: float


def fit(likelihood, p0, fixed: Sequence[int] = (0, 1), gtol: float = 1e-4,
        max_iter: int = 2000, errors: bool = True) -> FitResult:
    from scipy.optimize import minimize

    p0 = np.asarray(p0, dtype=np.float64).copy()
    free = np.array([k for k in range(len(p0)) if k not in set(fixed)], dtype=np.int64)
    calls = [0]

    def full(x):
        p = p0.copy()
        p[free] = x
        return p

    def fg(x):
        calls[0] += 1
        v, g = likelihood.nll_grad(full(x))
        return v, g[free]

    t0 = time.perf_counter()
    res = minimize(fg, p0[free], jac=True, method="BFGS",
                   options={"gtol": gtol, "maxiter": max_iter})
    p = full(res.x)
    err = None
    if errors:
        err = np.zeros_like(p)
        H = hessian(likelihood, p, free)
        try:
            cov = 2.0 * np.linalg.inv(H)
            err[free] = np.sqrt(np.clip(np.diag(cov), 0.0, None))
        except np.linalg.LinAlgError:
            err = None
    return FitResult(params=p, nll=float(res.fun), errors=err, n_calls=calls[0],
                     converged=bool(res.success), message=str(res.message),
                     seconds=time.perf_counter() - t0)


def hessian(likelihood, p, free, h: float = 1e-5) -> np.ndarray:
    """Symmetrised central-difference Hessian of -2 ln L over the free parameters."""
    n = len(free)
    H = np.empty((n, n))
    for a, k in enumerate(free):
        e = np.zeros_like(p)
        e[k] = h
        _, gp = likelihood.nll_grad(p + e)
        _, gm = likelihood.nll_grad(p - e)
        H[a] = (gp[free] - gm[free]) / (2 * h)
    return 0.5 * (H + H.T)
