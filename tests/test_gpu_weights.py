"""Weighted normalisation samples through the C ABI against the FP64 oracle.

With a weight w_j per normalisation point the integral is the weighted mean
sum_j w_j |A(y_j)|^2 / sum_j w_j (the paper's plain mean is w_j = 1). The
weights must follow their points through the set-time grouping by spline cell
and every evaluation path: computed and cached Breit-Wigner terms, the Re/Im
moments, the batched toys and the mass/width derivatives. Tolerances are those
of the unweighted tests (FP64 NLL 1e-12 relative, gradient 1e-8; FP32-mixed
NLL 1e-2 absolute and gradient 2e-5 at 10^6 events).
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, F64, Likelihood, MipwaError  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def weights_for(n, seed=3, lo=0.2, hi=3.0):
    return np.random.default_rng(seed).uniform(lo, hi, n)


def rel(a, b):
    return abs(a - b) / abs(b)


def grad_rel(g, gref):
    return np.linalg.norm(g - gref) / np.linalg.norm(gref)


def make(name, data, norm, w, mode=F64, on_device=False):
    lik = Likelihood(0, mode)
    lik.set_spec(P.spec_by_name(name))
    put = (lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(DEV)) if on_device else (
        lambda x: np.ascontiguousarray(x))
    lik.set_events(put(data))
    lik.set_norm_sample(put(norm), weights=None if w is None else put(w))
    return lik


@pytest.mark.parametrize("on_device", [False, True], ids=["host", "device"])
@pytest.mark.parametrize("name", ["pipipi_n10", "kpipi_n40", "kkk_n40"])
def test_fp64_weighted_matches_oracle(name, on_device):
    data, norm = P.data_sample(name, 20_000), P.uniform_sample(name, 30_000)
    w = weights_for(len(norm))
    p = synth.perturbed_params(P.spec_by_name(name), 5, 0.02)
    lik = make(name, data, norm, w, on_device=on_device)
    v, g = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm, norm_weights=w)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8
    assert rel(lik.nll(p), v) < 1e-13


def test_integer_weights_equal_repeated_points():
    name = "pipipi_n30"
    data, norm = P.data_sample(name, 10_000), P.uniform_sample(name, 20_000)
    k = np.random.default_rng(4).integers(0, 4, len(norm))
    p = synth.perturbed_params(P.spec_by_name(name), 6, 0.02)
    v, g = make(name, data, norm, k.astype(np.float64)).nll_grad(p)
    vr, gr = make(name, data, np.repeat(norm, k, axis=0), None).nll_grad(p)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-10


@pytest.mark.parametrize("cached", [False, True], ids=["computed", "cached"])
def test_fp32_weighted_1e6(cached):
    name = "pipipi_n40"
    n = 1_000_000
    data = P.data_sample(name, n, f32=True)
    norm = P.uniform_sample(name, n, f32=True)
    w = weights_for(n, seed=9).astype(np.float32)
    lik = make(name, data, norm, w, mode=F32, on_device=True)
    lik.enable_basis_cache(cached)
    spec = P.spec_by_name(name)
    for p in (synth.true_params(spec), synth.perturbed_params(spec, 4, 0.02)):
        v, g = lik.nll_grad(p)
        vr, gr = P.oracle_for(name).nll_grad(p, data.astype(np.float64), norm.astype(np.float64),
                                             norm_weights=w.astype(np.float64))
        assert abs(v - vr) < 1e-2, (v, vr)
        assert grad_rel(g, gr) < 2e-5


@pytest.mark.parametrize("mode", [F64, F32], ids=["fp64", "fp32"])
def test_reim_moments_weighted(mode):
    """The per-cell moments carry the weights: moment and direct
    normalisation agree and match the oracle."""
    name = "kpipi_n40_reim"
    f32 = mode == F32
    data = P.data_sample(name, 50_000, f32=f32)
    norm = P.uniform_sample(name, 200_000, f32=f32)
    w = weights_for(len(norm), seed=11).astype(norm.dtype)
    p = synth.perturbed_params(P.spec_by_name(name), 9, 0.02)
    lik = make(name, data, norm, w, mode=mode)
    vd, gd = lik.nll_grad(p)
    lik.enable_norm_gram(True)
    vg, gg = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data.astype(np.float64), norm.astype(np.float64),
                                         norm_weights=w.astype(np.float64))
    if f32:
        assert abs(vd - vr) < 1e-2 and abs(vg - vr) < 1e-2
        assert grad_rel(gd, gr) < 2e-5 and grad_rel(gg, gr) < 2e-5
    else:
        assert rel(vd, vr) < 1e-12 and rel(vg, vr) < 1e-12
        assert grad_rel(gd, gr) < 1e-8 and grad_rel(gg, gr) < 1e-8


@pytest.mark.parametrize("gram", [False, True], ids=["events", "moments"])
def test_toys_share_a_weighted_normalisation(gram):
    name = "pipipi_n30_reim" if gram else "pipipi_n30"
    sizes = [0, 1, 300, 5000, 257]
    spec = P.spec_by_name(name)
    pool = P.data_sample(name, sum(sizes), seed=5)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    norm = P.uniform_sample(name, 40_000)
    w = weights_for(len(norm), seed=12)
    params = np.stack([synth.perturbed_params(spec, 100 + t, 0.02) for t in range(len(sizes))])
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_norm_sample(torch.from_numpy(norm).to(DEV), weights=torch.from_numpy(w).to(DEV))
    lik.set_toys(torch.from_numpy(pool).to(DEV), offsets)
    lik.enable_norm_gram(gram)
    nll, grad = lik.nll_grad_toys(params)
    o = P.oracle_for(name)
    for t in range(len(sizes)):
        d = pool[offsets[t]:offsets[t + 1]]
        vr, gr = o.nll_grad(params[t], d, norm, norm_weights=w)
        assert abs(nll[t] - vr) <= 1e-12 * max(abs(vr), 1.0), (t, nll[t], vr)
        if sizes[t] == 0:
            assert np.all(grad[t] == 0.0)
        else:
            assert np.linalg.norm(grad[t] - gr) <= 1e-8 * np.linalg.norm(gr), t


def test_mass_width_derivatives_weighted():
    name = "pipipi_n10"
    spec = P.spec_by_name(name)
    data, norm = P.data_sample(name, 5000), P.uniform_sample(name, 8000)
    w = weights_for(len(norm), seed=13)
    p = synth.perturbed_params(spec, 7, 0.02)
    lik = make(name, data, norm, w)
    v, g, gbw = lik.nll_grad_bw(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm, norm_weights=w)
    assert rel(v, vr) < 1e-12 and grad_rel(g, gr) < 1e-8
    # d/dm_0 and d/dGamma_0 by five-point differences of the weighted oracle NLL
    m0, G0, L0 = spec.resonances[0]
    for which, h in ((0, 2e-6 * m0), (1, 2e-6 * G0)):
        def nll_at(d):
            res = list(spec.resonances)
            res[0] = (m0 + d, G0, L0) if which == 0 else (m0, G0 + d, L0)
            return oracle.Oracle(dataclasses.replace(spec, resonances=tuple(res))).nll(
                p, data, norm, norm_weights=w)
        fd = (-nll_at(2 * h) + 8 * nll_at(h) - 8 * nll_at(-h) + nll_at(-2 * h)) / (12 * h)
        np.testing.assert_allclose(gbw[which], fd, rtol=1e-5)


def test_weights_follow_a_new_knot_grid():
    name = "pipipi_n10"
    spec = P.spec_by_name(name)
    data, norm = P.data_sample(name, 8000), P.uniform_sample(name, 12_000)
    w = weights_for(len(norm), seed=14)
    lik = make(name, data, norm, w)
    knots = np.concatenate([np.linspace(spec.knots[0], 1.0, 6), np.linspace(1.3, spec.knots[-1], 7)])
    spec2 = synth.ModelSpec(name="nonuni", mD=spec.mD, m1=spec.m1, m2=spec.m2,
                            resonances=spec.resonances, knots=tuple(knots))
    lik.set_model(spec2.resonances, spec2.knots, spec2.r_res, spec2.r_D)
    p2 = synth.perturbed_params(spec2, 8, 0.02)
    v, g = lik.nll_grad(p2)
    vr, gr = oracle.Oracle(spec2).nll_grad(p2, data, norm, norm_weights=w)
    assert rel(v, vr) < 1e-12 and grad_rel(g, gr) < 1e-8


def test_weight_errors_keep_the_previous_sample():
    name = "pipipi_n10"
    data, norm = P.data_sample(name, 2000), P.uniform_sample(name, 3000)
    spec = P.spec_by_name(name)
    p = synth.perturbed_params(spec, 2, 0.02)
    w = weights_for(len(norm), seed=15)
    lik = make(name, data, norm, w)
    v0, _ = lik.nll_grad(p)
    bad = w.copy()
    bad[17] = np.nan
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.set_norm_sample(norm[::-1].copy(), weights=bad)
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.set_norm_sample(norm, weights=np.zeros(len(norm)))
    with pytest.raises(ValueError):
        lik.set_norm_sample(norm, weights=w[:-1])
    assert lik.nll_grad(p)[0] == v0
    # negative weights are allowed while the sum stays positive
    wn = w.copy()
    wn[::7] *= -0.25
    lik.set_norm_sample(norm, weights=wn)
    vr, _ = P.oracle_for(name).nll_grad(p, data, norm, norm_weights=wn)
    assert rel(lik.nll_grad(p)[0], vr) < 1e-12
    # without weights again: the plain mean
    lik.set_norm_sample(norm)
    vr, _ = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(lik.nll_grad(p)[0], vr) < 1e-12
