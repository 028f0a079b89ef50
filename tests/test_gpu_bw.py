"""Free Breit-Wigner masses and widths: mipwa_set_resonances and the analytic
d NLL / d(m_r, Gamma_r) of mipwa_nll_grad_bw against central differences of
the FP64 oracle's -2 ln L in the masses and widths (the oracle evaluates the
plain definition at each shifted resonance)."""
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


def with_res(spec, res):
    return dataclasses.replace(spec, resonances=tuple(res))


def oracle_bw_derivs(spec, p, data, norm, rel_h=2e-6):
    """Five-point central differences of the oracle NLL in every m_r, Gamma_r."""
    out = []
    for r, (m, w, L) in enumerate(spec.resonances):
        for which, x in ((0, m), (1, w)):
            h = rel_h * x
            vals = []
            for k in (-2, -1, 1, 2):
                res = list(spec.resonances)
                mm, ww = (m + k * h, w) if which == 0 else (m, w + k * h)
                res[r] = (mm, ww, L)
                vals.append(oracle.Oracle(with_res(spec, res)).nll(p, data, norm))
            out.append((vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * h))
    return np.array(out)


SPIN0 = synth.ModelSpec(name="s0", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                        resonances=((0.775, 0.149, 1), (0.98, 0.06, 0), (1.275, 0.185, 2)),
                        knots=synth.uniform_knots(0.078, 2.987, 12))


@pytest.mark.parametrize("spec", [synth.pipipi(10), synth.kpipi(12), SPIN0,
                                  synth.as_reim(synth.pipipi(10))], ids=lambda s: s.name)
def test_bw_derivatives_match_oracle_differences(spec):
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    dens = synth.numpy_density(lambda x: o.density(truth, x))
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    data = synth.accept_reject(spec, 3000, dens, seed=17).numpy()
    norm = synth.grid_in_plot(spec, 50, ins).numpy()
    p = synth.perturbed_params(spec, 19, 0.02)
    lik = Likelihood(0, F32)  # the call computes in FP64 whatever the mode
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    v, g, gbw = lik.nll_grad_bw(p)
    vr, gr = o.nll_grad(p, data, norm)
    assert abs(v - vr) <= 1e-12 * abs(vr)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)
    fd = oracle_bw_derivs(spec, p, data, norm)
    assert np.abs(gbw - fd).max() <= 1e-6 * np.abs(fd).max(), (gbw, fd)
    for r in range(spec.n_res):  # each derivative, not only the largest
        np.testing.assert_allclose(gbw[2 * r:2 * r + 2], fd[2 * r:2 * r + 2], rtol=1e-5,
                                   atol=1e-7 * np.abs(fd).max())


def test_set_resonances_keeps_samples_and_rebuilds_caches():
    name = "kpipi_n40"
    spec = P.spec_by_name(name)
    data, norm = P.data_sample(name, 20_000), P.uniform_sample(name, 30_000)
    p = synth.perturbed_params(spec, 5)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    lik.enable_basis_cache(True)
    lik.nll_grad(p)  # builds the cache for the old resonances
    res2 = [(m * 1.01, w * 0.9, L) for (m, w, L) in spec.resonances]
    lik.set_resonances(res2)
    v, g = lik.nll_grad(p)
    vr, gr = oracle.Oracle(with_res(spec, res2)).nll_grad(p, data, norm)
    assert abs(v - vr) <= 1e-12 * abs(vr)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.set_resonances(res2[:1])
    fresh = Likelihood(0, F64)
    with pytest.raises(MipwaError, match="ESTATE"):
        fresh.set_resonances(res2)


def test_set_resonances_rebuilds_moments():
    name = "pipipi_n10_reim"
    spec = P.spec_by_name(name)
    data, norm = P.data_sample(name, 5000), P.uniform_sample(name, 20_000)
    p = synth.perturbed_params(spec, 6, 0.02)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    lik.enable_norm_gram(True)
    lik.nll_grad(p)
    res2 = [(m * 0.99, w * 1.1, L) for (m, w, L) in spec.resonances]
    lik.set_resonances(res2)
    v, g = lik.nll_grad(p)
    vr, gr = oracle.Oracle(with_res(spec, res2)).nll_grad(p, data, norm)
    assert abs(v - vr) <= 1e-12 * abs(vr)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)


def test_fit_with_free_rho_mass_and_width():
    """A toy drawn at the true rho(770) mass and width, fitted with both free
    (started 5 MeV and 10 MeV off): the fit converges near the truth."""
    from paper_1703_03284_gb300.fit import FreeResonances, fit

    name = "pipipi_n10"
    spec = P.spec_by_name(name)
    data = P.data_sample(name, 100_000, seed=3)
    norm = P.grid_sample(name, 300)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    truth = synth.true_params(spec)
    (m0, w0, L0), (m1, w1, L1) = spec.resonances
    x0 = np.concatenate([truth, [m0 + 0.005, w0 - 0.010, m1, w1]])
    free = FreeResonances(lik, [L0, L1])
    P_ = spec.n_params
    res = fit(free, x0, fixed=(0, 1, P_ + 2, P_ + 3))
    assert res.converged, (res.message, res.edm)
    for k, want in ((P_, m0), (P_ + 1, w0)):
        assert abs(res.params[k] - want) < 5 * res.errors[k], (k, res.params[k], want, res.errors[k])
        assert 0 < res.errors[k] < 0.01


def test_isobar_baseline_matches_oracle_and_fits():
    """Isobar S-wave baseline: two scalar Breit-Wigner terms in place of the
    spline (knot values held at zero). FP64 parity with the oracle, then a fit
    of the coefficients from a perturbed start with the spline fixed."""
    from paper_1703_03284_gb300.fit import fit

    spec = synth.pipipi_isobar()
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    dens = synth.numpy_density(lambda x: o.density(truth, x))
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    data = synth.accept_reject(spec, 50_000, dens, seed=23).numpy()
    norm = synth.grid_in_plot(spec, 200, ins).numpy()
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    p = truth.copy()
    p[2:8] += 0.01 * np.random.default_rng(4).standard_normal(6)
    v, g = lik.nll_grad(p)
    vr, gr = o.nll_grad(p, data, norm)
    assert abs(v - vr) <= 1e-12 * abs(vr)
    assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)
    res = fit(lik, p, fixed=spec.fixed)
    assert res.converged, (res.message, res.edm)
    free = np.arange(2, 8)
    assert np.all(np.abs(res.params[free] - truth[free]) < 5 * res.errors[free])
    assert np.all(res.params[8:] == 0.0)
