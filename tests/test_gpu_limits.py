"""The library at its size limits: 4 resonances and 64 knots (the maximum),
2 knots (one spline segment, no interior second derivative), and the
arguments one past the limits."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, F64, Likelihood, MipwaError  # noqa: E402

DEV = "cuda:0"

# rho(770) P, f0(980) S, f2(1270) D, rho(1450) P
RES4 = ((0.77526, 0.1491, 1), (0.98, 0.06, 0), (1.2755, 0.1867, 2), (1.465, 0.4, 1))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def spec_of(n_knots, res=RES4, form="magphase"):
    return synth.ModelSpec(name=f"lim_{n_knots}_{len(res)}", mD=synth.M_D, m1=synth.M_PI,
                           m2=synth.M_PI, resonances=res,
                           knots=synth.uniform_knots(0.078, 2.987, n_knots), swave_form=form)


def sample(spec, n, seed, f32):
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    dens = synth.numpy_density(lambda x: o.density(truth, x))
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    dt = torch.float32 if f32 else torch.float64
    data = synth.accept_reject(spec, n, dens, seed=seed, dtype=dt).numpy()
    norm = synth.uniform_in_plot(spec, n, ins, seed=seed + 1, dtype=dt).numpy()
    return o, data, norm


def check(spec, mode, n, gram=False, seed=11):
    f32 = mode == F32
    o, data, norm = sample(spec, n, seed, f32)
    lik = Likelihood(0, mode)
    lik.set_spec(spec)
    lik.set_events(torch.from_numpy(data).to(DEV))
    lik.set_norm_sample(torch.from_numpy(norm).to(DEV))
    lik.enable_norm_gram(gram)
    p = synth.perturbed_params(spec, seed + 2, 0.02)
    v, g = lik.nll_grad(p)
    vr, gr = o.nll_grad(p, data.astype(np.float64), norm.astype(np.float64))
    if f32:
        assert abs(v - vr) < 1e-2, (v, vr)
        assert np.linalg.norm(g - gr) < 2e-5 * np.linalg.norm(gr)
    else:
        assert abs(v - vr) <= 1e-12 * abs(vr), (v, vr)
        assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)
    return lik, p, o, data, norm


@pytest.mark.parametrize("mode", [F64, F32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("form,gram", [("magphase", False), ("reim", False), ("reim", True)],
                         ids=["magphase", "reim", "reim-moments"])
def test_maximum_model(mode, form, gram):
    """64 knots (63 segments, 3969 cells) and 4 resonances: every table at its
    largest (moments: 94 per cell)."""
    check(spec_of(64, RES4, form), mode, 200_000, gram)


@pytest.mark.parametrize("mode", [F64, F32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("form,gram", [("magphase", False), ("reim", True)],
                         ids=["magphase", "reim-moments"])
def test_two_knots(mode, form, gram):
    """Two knots: one segment continued over the whole plot, a linear spline."""
    check(spec_of(2, RES4[:2], form), mode, 50_000, gram)


def test_bw_derivatives_at_four_resonances():
    spec = spec_of(64)
    o, data, norm = sample(spec, 3000, 21, False)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    p = synth.perturbed_params(spec, 5, 0.02)
    v, g, gbw = lik.nll_grad_bw(p)
    h = 2e-6
    for r in range(4):
        m, w, L = spec.resonances[r]
        vals = []
        for k in (-1, 1):
            res = list(spec.resonances)
            res[r] = (m * (1 + k * h), w, L)
            vals.append(oracle.Oracle(dataclasses.replace(spec, resonances=tuple(res))).nll(p, data, norm))
        fd = (vals[1] - vals[0]) / (2 * h * m)
        assert abs(gbw[2 * r] - fd) <= 1e-5 * max(abs(fd), 1.0), (r, gbw[2 * r], fd)


def test_arguments_past_the_limits():
    lik = Likelihood(0, F64)
    lik.set_masses(synth.M_D, synth.M_PI, synth.M_PI)
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.set_model(RES4, synth.uniform_knots(0.078, 2.987, 65), 1.5, 5.0)
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.set_model(RES4 + ((1.5, 0.1, 0),), synth.uniform_knots(0.078, 2.987, 10), 1.5, 5.0)
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.set_model(RES4, (1.0,), 1.5, 5.0)
    lik.set_model(RES4, synth.uniform_knots(0.078, 2.987, 64), 1.5, 5.0)
    assert lik.num_params() == 2 * 4 + 2 * 64
