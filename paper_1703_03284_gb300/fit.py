"""Host quasi-Newton minimiser of -2 ln L (the unbinned maximum-likelihood fit
of arXiv:1703.03284, Sec. 2), calling the library's NLL+gradient each step.

Fixed parameters (by default Re c_0, Im c_0: the reference wave) are held at
their start values. The fit is BFGS on the analytic gradient, followed by
Newton steps with the Hessian of -2 ln L (central differences of the analytic
gradient), which pin the minimum by the gradient alone: near the minimum the
change of -2 ln L between nearby points is below its own rounding in FP32, so
a line search on function values stalls there while the gradient stays exact
to ~1e-6. Uncertainties: cov = 2 H^{-1}.
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
    edm: float  # estimated distance to the minimum in units of sigma: max |g_k| sigma_k / 2


def fit(likelihood, p0, fixed: Sequence[int] = (0, 1), gtol: float = 1e-3,
        max_iter: int = 2000, newton_steps: int = 10, edm_tol: float = 1e-3) -> FitResult:
    from scipy.optimize import minimize

    p0 = np.asarray(p0, dtype=np.float64).copy()
    fixed = set(int(k) for k in fixed)
    free = np.array([k for k in range(len(p0)) if k not in fixed], dtype=np.int64)
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
    message = str(res.message)
    H = hessian(likelihood, p, free)
    calls[0] += 2 * len(free)
    err = np.zeros_like(p)
    edm = np.inf
    steps_h = None
    for it in range(newton_steps + 1):
        try:
            Hinv = np.linalg.inv(H)
        except np.linalg.LinAlgError:
            message += "; singular Hessian"
            break
        sig = np.sqrt(np.clip(np.diag(2.0 * Hinv), 0.0, None))
        if steps_h is None:
            # once the scale of each parameter is known, difference the gradient
            # over a tenth of its uncertainty (well above FP32 gradient noise)
            steps_h = np.maximum(0.1 * sig, 1e-7)
            H = hessian(likelihood, p, free, h=steps_h)
            calls[0] += 2 * len(free)
            continue
        _, g = likelihood.nll_grad(p)
        calls[0] += 1
        edm = float(np.max(np.abs(g[free]) * sig) / 2.0)
        err[free] = sig
        if edm < edm_tol:
            break
        p[free] -= Hinv @ g[free]
    v, _ = likelihood.nll_grad(p)
    calls[0] += 1
    converged = bool(edm < edm_tol)
    return FitResult(params=p, nll=float(v), errors=err, n_calls=calls[0], converged=converged,
                     message=message, seconds=time.perf_counter() - t0, edm=edm)


def hessian(likelihood, p, free, h=1e-5) -> np.ndarray:
    """Symmetrised central-difference Hessian of -2 ln L over the free
    parameters; h is one step for all of them or one per free parameter."""
    n = len(free)
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    H = np.empty((n, n))
    for a, k in enumerate(free):
        e = np.zeros_like(p)
        e[k] = hs[a]
        _, gp = likelihood.nll_grad(p + e)
        _, gm = likelihood.nll_grad(p - e)
        H[a] = (gp[free] - gm[free]) / (2 * hs[a])
    return 0.5 * (H + H.T)
