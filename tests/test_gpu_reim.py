"""The Re/Im (complex-plane) S-wave form and its moment normalisation against
the FP64 oracle, through the C ABI.

The oracle evaluates the normalisation integral as the plain sample mean of
|A|^2; the library either does the same (direct) or forms it from per-cell
moments of the normalisation sample (gram). Tolerances are those of the
magnitude/phase form: FP64 NLL 1e-12 relative and gradient 1e-8 norm-wise;
FP32-mixed NLL 1e-2 absolute and gradient 2e-5 at 10^6 events.
"""
import numpy as np
import pytest
import torch

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


def make(name, data, norm, mode=F64, gram=False):
    lik = Likelihood(0, mode)
    lik.set_spec(P.spec_by_name(name))
    lik.set_events(torch.from_numpy(np.ascontiguousarray(data)).to(DEV))
    lik.set_norm_sample(torch.from_numpy(np.ascontiguousarray(norm)).to(DEV))
    lik.enable_norm_gram(gram)
    return lik


def rel(a, b):
    return abs(a - b) / abs(b)


def grad_rel(g, gref):
    return np.linalg.norm(g - gref) / np.linalg.norm(gref)


@pytest.mark.parametrize("gram", [False, True], ids=["direct", "gram"])
@pytest.mark.parametrize("name", ["pipipi_n30_reim", "kpipi_n40_reim", "kkk_n40_reim"])
def test_reim_fp64_matches_oracle(name, gram):
    data, norm = P.data_sample(name, 20_000), P.uniform_sample(name, 30_000)
    spec = P.spec_by_name(name)
    p = synth.perturbed_params(spec, 5, 0.02)
    lik = make(name, data, norm, gram=gram)
    v, g = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8
    assert rel(lik.nll(p), v) < 1e-13


@pytest.mark.parametrize("nd,nn", [(1, 1), (255, 257), (0, 300), (1023, 2), (5000, 4097)])
def test_reim_gram_ragged_sizes(nd, nn):
    name = "pipipi_n10_reim"
    data = P.data_sample(name, 6000)[:nd]
    norm = P.uniform_sample(name, 5000)[:nn]
    p = synth.perturbed_params(P.spec_by_name(name), 7, 0.02)
    lik = make(name, data, norm, gram=True)
    v, g = lik.nll_grad(p)
    if nd == 0:
        assert v == 0.0 and np.all(g == 0.0)
        return
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8


def test_reim_gram_grid_normalisation_and_model_change():
    """Normalisation on the evenly spaced grid (Sec. 4), then a different knot
    grid and a spin-0 resonance: the moments follow the model."""
    name = "pipipi_n10_reim"
    spec = P.spec_by_name(name)
    data, norm = P.data_sample(name, 10_000), P.grid_sample(name, 100)
    p = synth.perturbed_params(spec, 3, 0.02)
    lik = make(name, data, norm, gram=True)
    v, g = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12 and grad_rel(g, gr) < 1e-8
    import oracle
    knots = np.concatenate([np.linspace(spec.knots[0], 1.0, 6), np.linspace(1.3, spec.knots[-1], 7)])
    spec2 = synth.ModelSpec(name="nonuni", mD=spec.mD, m1=spec.m1, m2=spec.m2,
                            resonances=spec.resonances + ((0.98, 0.06, 0),),
                            knots=tuple(knots), swave_form="reim")
    lik.set_model(spec2.resonances, spec2.knots, spec2.r_res, spec2.r_D)
    p2 = synth.perturbed_params(spec2, 8, 0.02)
    v2, g2 = lik.nll_grad(p2)
    vr2, gr2 = oracle.Oracle(spec2).nll_grad(p2, data, norm)
    assert rel(v2, vr2) < 1e-12 and grad_rel(g2, gr2) < 1e-8


def test_reim_gram_equals_direct_and_is_deterministic():
    name = "kpipi_n40_reim"
    data, norm = P.data_sample(name, 50_000), P.uniform_sample(name, 200_000)
    p = synth.perturbed_params(P.spec_by_name(name), 9, 0.02)
    lik = make(name, data, norm, gram=False)
    vd, gd = lik.nll_grad(p)
    lik.enable_norm_gram(True)
    lik.build_norm_gram()
    vg, gg = lik.nll_grad(p)
    assert rel(vg, vd) < 1e-12
    assert grad_rel(gg, gd) < 1e-10
    # the NLL is bitwise reproducible; the spline adjoint's shared-memory bins
    # are summed in arrival order, so the gradient repeats to rounding
    vg2, gg2 = lik.nll_grad(p)
    assert vg2 == vg
    np.testing.assert_allclose(gg2, gg, rtol=1e-13, atol=1e-13 * np.abs(gg).max())


@pytest.mark.parametrize("gram", [False, True], ids=["direct", "gram"])
@pytest.mark.parametrize("cached", [False, True], ids=["computed", "cached"])
def test_reim_fp32_1e6(gram, cached):
    name = "pipipi_n40_reim"
    n = 1_000_000
    data = P.data_sample(name, n, f32=True)
    norm = P.uniform_sample(name, n, f32=True)
    spec = P.spec_by_name(name)
    lik = make(name, data, norm, mode=F32, gram=gram)
    lik.enable_basis_cache(cached)
    d64, n64 = data.astype(np.float64), norm.astype(np.float64)
    for p in (synth.true_params(spec), synth.perturbed_params(spec, 4, 0.02)):
        v, g = lik.nll_grad(p)
        vr, gr = P.oracle_for(name).nll_grad(p, d64, n64)
        assert abs(v - vr) < 1e-2, (v, vr)
        assert grad_rel(g, gr) < 2e-5


def test_reim_amp2_per_event():
    name = "kpipi_n40_reim"
    spec = P.spec_by_name(name)
    o = P.oracle_for(name)
    ev = P.uniform_sample(name, 100_000)
    p = synth.perturbed_params(spec, 2, 0.02)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    got = lik.amp2(p, torch.from_numpy(ev).to(DEV)).cpu().numpy()
    np.testing.assert_allclose(got, o.amp2(p, ev), rtol=1e-12, atol=0)


def test_reim_form_errors():
    name = "pipipi_n10"
    data, norm = P.data_sample(name, 1000), P.uniform_sample(name, 1000)
    lik = make(name, data, norm)
    with pytest.raises(MipwaError):
        lik.set_swave_form(2)
    lik.enable_norm_gram(True)  # magnitude/phase form: evaluations refuse
    p = synth.true_params(P.spec_by_name(name))
    with pytest.raises(MipwaError, match="ESTATE"):
        lik.nll_grad(p)
    with pytest.raises(MipwaError, match="ESTATE"):
        lik.build_norm_gram()
    lik.enable_norm_gram(False)
    v, _ = lik.nll_grad(p)
    vr, _ = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12


@pytest.mark.parametrize("mode", [F64, F32], ids=["fp64", "fp32"])
def test_reim_toys_with_gram(mode):
    """Batched toys sharing one normalisation sample: with the moments, each
    toy's normalisation costs O(cells); every toy matches the oracle."""
    name = "pipipi_n30_reim"
    f32 = mode == F32
    sizes = [0, 1, 300, 5000, 257, 20000]
    spec = P.spec_by_name(name)
    pool = P.data_sample(name, sum(sizes), seed=5, f32=f32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    norm = P.uniform_sample(name, 40_000, f32=f32)
    params = np.stack([synth.perturbed_params(spec, 100 + t, 0.02) for t in range(len(sizes))])
    lik = Likelihood(0, mode)
    lik.set_spec(spec)
    lik.set_norm_sample(torch.from_numpy(norm).to(DEV))
    lik.set_toys(torch.from_numpy(pool).to(DEV), offsets)
    lik.enable_norm_gram(True)
    lik.enable_basis_cache(f32)
    nll, grad = lik.nll_grad_toys(params)
    o = P.oracle_for(name)
    for t in range(len(sizes)):
        d = pool[offsets[t]:offsets[t + 1]].astype(np.float64)
        vr, gr = o.nll_grad(params[t], d, norm.astype(np.float64))
        if f32:
            assert abs(nll[t] - vr) < 1e-2, (t, nll[t], vr)
        else:
            assert abs(nll[t] - vr) <= 1e-12 * max(abs(vr), 1.0), (t, nll[t], vr)
        if sizes[t] == 0:
            assert np.all(grad[t] == 0.0)
        else:
            tol = 2e-5 if f32 else 1e-8
            assert np.linalg.norm(grad[t] - gr) <= tol * np.linalg.norm(gr), t
    nll2, _ = lik.nll_grad_toys(params)
    np.testing.assert_array_equal(nll2, nll)
