"""The host quasi-Newton fit (paper_1703_03284_gb300.fit) and toy pulls.

CPU: the minimiser driven by the oracle on a small toy (host logic only).
GPU: the full fit of 10^6 + 10^6 events with 30 knots through the library,
FP64 and FP32-mixed, and the FP32 fit within 0.05 sigma of the FP64 fit.
"""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P


class OracleLikelihood:
    """The oracle behind the nll_grad(params) interface the minimiser uses."""

    def __init__(self, name, data, norm):
        self.o = P.oracle_for(name)
        self.data, self.norm = data, norm

    def nll_grad(self, p):
        return self.o.nll_grad(p, self.data, self.norm)


def test_fit_converges_on_oracle_toy():
    """From the truth, BFGS reaches a minimum whose -2 ln L gain over the truth
    is chi-square-like for the free parameters, with finite positive errors;
    the fixed reference coefficient stays put."""
    from paper_1703_03284_gb300.fit import fit

    name = "pipipi_n10"
    spec = P.spec_by_name(name)
    data = P.data_sample(name, 20_000, seed=31)
    norm = P.grid_sample(name, 200)
    lik = OracleLikelihood(name, data, norm)
    truth = synth.true_params(spec)
    res = fit(lik, truth, fixed=(0, 1))
    assert res.converged, (res.message, res.edm)
    free = np.arange(2, spec.n_params)
    k = len(free)
    gain = lik.nll_grad(truth)[0] - res.nll
    assert 0.0 <= gain < k + 5 * np.sqrt(2 * k)
    assert np.all(np.isfinite(res.errors[free])) and np.all(res.errors[free] > 0)
    assert res.params[0] == truth[0] and res.params[1] == truth[1]
    _, g = lik.nll_grad(res.params)
    assert np.abs(g[free]).max() < 1e-2


@pytest.mark.gpu
def test_full_fit_fp32_within_005_sigma_of_fp64():
    from paper_1703_03284_gb300 import F32, F64, Likelihood
    from paper_1703_03284_gb300.fit import fit

    name = "pipipi_n30"
    spec = P.spec_by_name(name)
    data = torch.from_numpy(P.data_sample(name, 1_000_000, f32=True)).to("cuda:0")
    norm = torch.from_numpy(P.uniform_sample(name, 1_000_000, f32=True)).to("cuda:0")
    start = synth.perturbed_params(spec, 21, 0.03)
    fits = {}
    for mode in (F64, F32):
        lik = Likelihood(0, mode)
        lik.set_spec(spec)
        lik.set_events(data)
        lik.set_norm_sample(norm)
        fits[mode] = fit(lik, start, fixed=(0, 1))
        assert fits[mode].converged, (fits[mode].message, fits[mode].edm)
    f64, f32 = fits[F64], fits[F32]
    free = np.arange(2, spec.n_params)
    shift = np.abs(f32.params[free] - f64.params[free]) / f64.errors[free]
    assert shift.max() < 0.05, shift.max()
    # the FP64 minimum is a stationary point of the oracle's -2 ln L too
    o = P.oracle_for(name)
    _, g = o.nll_grad(f64.params, data.cpu().numpy().astype(np.float64),
                      norm.cpu().numpy().astype(np.float64))
    assert np.abs(g[free] * f64.errors[free]).max() < 1e-2
