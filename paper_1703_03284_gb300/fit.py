"""Host quasi-Newton minimiser of -2 ln L (the unbinned maximum-likelihood fit
of arXiv:1703.03284, Sec. 2), calling the library's NLL+gradient each step.

Fixed parameters (by default Re c_0, Im c_0: the reference wave) are held at
their start values. The fit runs in three stages:

1. a second-derivative estimate at the start point (central differences of the
   analytic gradient), whose eigenvalues, taken in absolute value and floored,
   whiten the free parameters, so that -2 ln L has roughly unit curvature in
   every direction (the start-up estimate of a variable-metric minimiser);
2. BFGS on the analytic gradient in the whitened coordinates;
3. Newton steps with the Hessian of -2 ln L differenced over a tenth of each
   parameter's uncertainty, which pin the minimum by the gradient alone: near
   the minimum the change of -2 ln L between nearby points is below its own
   rounding in FP32, so a line search on function values stalls there while
   the gradient stays exact to ~1e-6.

Uncertainties: cov = 2 H^{-1}.
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
    W = whitening(likelihood, p0, free)
    calls[0] += 2 * len(free)

    def fg_white(y):
        v, g = fg(p0[free] + W @ y)
        return v, W.T @ g

    res = minimize(fg_white, np.zeros(len(free)), jac=True, method="BFGS",
                   options={"gtol": gtol, "maxiter": max_iter})
    p = full(p0[free] + W @ res.x)
    message = str(res.message)
    # difference the gradient over a tenth of each parameter's uncertainty at
    # the start (well above FP32 gradient noise): sigma^2 = 2 (W W^T)_kk
    steps_h = np.maximum(0.1 * np.sqrt(2.0 * np.sum(W * W, axis=1)), 1e-7)
    H = hessian(likelihood, p, free, h=steps_h)
    calls[0] += 2 * len(free)
    err = np.zeros_like(p)
    edm = np.inf
    for it in range(newton_steps + 1):
        try:
            Hinv = np.linalg.inv(H)
        except np.linalg.LinAlgError:
            message += "; singular Hessian"
            break
        sig = np.sqrt(np.clip(np.diag(2.0 * Hinv), 0.0, None))
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


def whitening(likelihood, p, free, floor: float = 1e-6) -> np.ndarray:
    """W with W^T H W ~ 1 for the second-derivative matrix H of -2 ln L at p:
    W = V |Lambda|^{-1/2} from the eigen-decomposition of H, the eigenvalues
    taken in absolute value (a start point need not lie where -2 ln L is
    convex) and floored at `floor` times the largest one."""
    h = 1e-4 * np.maximum(1.0, np.abs(p[free]))
    H = hessian(likelihood, p, free, h=h)
    lam, V = np.linalg.eigh(H)
    lam = np.abs(lam)
    lam = np.maximum(lam, floor * max(lam.max(), 1e-300))
    return V / np.sqrt(lam)


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


class FreeResonances:
    """-2 ln L over [params..., m_0, Gamma_0, ..., m_{R-1}, Gamma_{R-1}] for fits
    in which the Breit-Wigner masses and widths float too (Sec. 2 holds them
    fixed): each call sets the resonances and evaluates the NLL with its
    gradient with respect to all of them (FP64)."""

    def __init__(self, likelihood, spins):
        self.lik = likelihood
        self.spins = [int(s) for s in spins]

    def nll_grad(self, x):
        x = np.asarray(x, dtype=np.float64)
        R = len(self.spins)
        p, bw = x[: len(x) - 2 * R], x[len(x) - 2 * R:]
        self.lik.set_resonances([(bw[2 * r], bw[2 * r + 1], self.spins[r]) for r in range(R)])
        v, g, gbw = self.lik.nll_grad_bw(p)
        return v, np.concatenate([g, gbw])
