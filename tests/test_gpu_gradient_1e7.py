"""FP64 gradient of -2 ln L at the differentiation workload's size: 10^7 data
events (accept-reject from the model's |A|^2) and 10^7 uniform phase-space
normalisation events, 40 knots, for D+ -> pi- pi+ pi+ (rho, f2) and
D+ -> K- pi+ pi+ (K*(892), K2*(1430)).

The library's analytic gradient (the adjoint kernel, amplitudes recomputed)
is checked against the oracle's gradient (1e-8 norm-wise relative) and, for a
subset of parameters that touches every part of the adjoint (an imaginary and
a real BW coefficient, knot magnitudes and phases at both ends and inside),
against central differences of the oracle's own -2 ln L with step 1e-6. The
difference tolerance is the truncation term (1e-6 relative) plus the rounding
term of a difference quotient, 50 eps |NLL| / h.
"""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_1703_03284_gb300 import F64, Likelihood  # noqa: E402

N = 10_000_000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("name", ["pipipi_n40", "kpipi_n40"])
def test_fp64_gradient_1e7(name):
    spec = P.spec_by_name(name)
    o = P.oracle_for(name)
    data = P.data_sample(name, N, seed=41)
    norm = P.uniform_sample(name, N, seed=42)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(torch.from_numpy(data).to("cuda:0"))
    lik.set_norm_sample(torch.from_numpy(norm).to("cuda:0"))
    p = synth.perturbed_params(spec, 17)
    v, g = lik.nll_grad(p)
    vr, gr = o.nll_grad(p, data, norm)
    assert abs(v - vr) <= 1e-12 * abs(vr), (v, vr)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr), np.abs(g - gr).max()
    R, K = spec.n_res, spec.n_knots
    h = 1e-6
    subset = [3, 2, 2 * R, 2 * R + K // 2, 2 * R + K - 1, 2 * R + K, 2 * R + K + 7,
              2 * R + 2 * K - 1]
    for k in subset:
        e = np.zeros_like(p)
        e[k] = h
        fd = (o.nll(p + e, data, norm) - o.nll(p - e, data, norm)) / (2 * h)
        tol = 1e-6 * abs(g[k]) + 50 * np.finfo(float).eps * abs(vr) / h
        assert abs(g[k] - fd) <= tol, (k, g[k], fd, tol)
