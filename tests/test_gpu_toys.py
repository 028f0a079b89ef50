"""Batched toys (one launch for many toy samples sharing a normalisation
sample) against the oracle, toy by toy."""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, F64, Likelihood  # noqa: E402

SIZES = [0, 1, 300, 5000, 257, 20000]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def toy_problem(name, f32):
    spec = P.spec_by_name(name)
    pool = P.data_sample(name, sum(SIZES), seed=5, f32=f32)
    offsets = np.concatenate([[0], np.cumsum(SIZES)]).astype(np.int64)
    norm = P.uniform_sample(name, 40_000, f32=f32)
    params = np.stack([synth.perturbed_params(spec, 100 + t) for t in range(len(SIZES))])
    return spec, pool, offsets, norm, params


def make_toys(name, pool, offsets, norm, mode, cached=False, graph=True):
    lik = Likelihood(0, mode)
    lik.set_spec(P.spec_by_name(name))
    lik.set_norm_sample(torch.from_numpy(norm).to("cuda:0"))
    lik.set_toys(torch.from_numpy(pool).to("cuda:0"), offsets)
    lik.enable_basis_cache(cached)
    lik.set_toys_graph(graph)
    return lik


@pytest.mark.parametrize("cached", [False, True], ids=["direct", "cached"])
@pytest.mark.parametrize("graph", [True, False], ids=["graph", "nograph"])
def test_toys_fp64_match_oracle(cached, graph):
    name = "pipipi_n30"
    spec, pool, offsets, norm, params = toy_problem(name, False)
    lik = make_toys(name, pool, offsets, norm, F64, cached, graph)
    nll, grad = lik.nll_grad_toys(params)
    o = P.oracle_for(name)
    for t in range(len(SIZES)):
        d = pool[offsets[t]:offsets[t + 1]]
        vr, gr = o.nll_grad(params[t], d, norm)
        assert abs(nll[t] - vr) <= 1e-12 * max(abs(vr), 1.0), (t, nll[t], vr)
        if SIZES[t] == 0:
            assert np.all(grad[t] == 0.0)
        else:
            assert np.linalg.norm(grad[t] - gr) <= 1e-8 * np.linalg.norm(gr), t
    # repeat: the work queue and the flags are reset by the launch itself
    nll2, grad2 = lik.nll_grad_toys(params)
    np.testing.assert_allclose(nll2, nll, rtol=1e-14, atol=1e-9)


def test_toys_fp32_match_oracle_and_autotune():
    name = "kpipi_n40"
    spec, pool, offsets, norm, params = toy_problem(name, True)
    lik = make_toys(name, pool, offsets, norm, F32, cached=True)
    nll, grad = lik.nll_grad_toys(params)
    o = P.oracle_for(name)
    for t in range(len(SIZES)):
        d = pool[offsets[t]:offsets[t + 1]].astype(np.float64)
        vr, gr = o.nll_grad(params[t], d, norm.astype(np.float64))
        assert abs(nll[t] - vr) < 1e-2, (t, nll[t], vr)
        if SIZES[t] > 0:
            assert np.linalg.norm(grad[t] - gr) <= 1e-5 * np.linalg.norm(gr), t
    best = lik.toys_autotune(params)
    assert best in (65536, 131072, 262144, 524288, 1048576, 2097152)
    nll2, grad2 = lik.nll_grad_toys(params)
    np.testing.assert_allclose(nll2, nll, rtol=0, atol=1e-3)


def test_toys_equal_single_fits():
    """Each toy of the batched launch equals a single-sample evaluation."""
    name = "pipipi_n10"
    spec, pool, offsets, norm, params = toy_problem(name, False)
    lik = make_toys(name, pool, offsets, norm, F64)
    nll, grad = lik.nll_grad_toys(params)
    single = Likelihood(0, F64)
    single.set_spec(spec)
    single.set_norm_sample(norm)
    for t in range(len(SIZES)):
        single.set_events(pool[offsets[t]:offsets[t + 1]])
        v, g = single.nll_grad(params[t])
        assert abs(nll[t] - v) <= 1e-12 * max(abs(v), 1.0)
        np.testing.assert_allclose(grad[t], g, rtol=1e-9, atol=1e-9 * (np.abs(g).max() + 1))
