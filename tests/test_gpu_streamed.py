"""The pipelined call (mipwa_nll_grad_streamed): both samples copied from host
memory in pieces, each piece checked, grouped by cell and evaluated as it
lands, one combine at the end. Checked against the oracle (FP64: NLL 1e-12
relative, gradient 1e-8; FP32: NLL 1e-2 absolute, gradient 2e-5), against the
set_events + set_norm_sample + nll_grad path on the same samples, and for the
state it leaves: the stored samples (permutations of the inputs, usable by
the other calls, regrouped as a whole before the moment normalisation) and an
unchanged state when an event lies outside the plot."""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, F64, Likelihood, MipwaError  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def rows_sorted(a):
    a = np.asarray(a)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def check(v, g, vr, gr, f32):
    if f32:
        assert abs(v - vr) < 1e-2, (v, vr)
        assert np.linalg.norm(g - gr) <= 2e-5 * np.linalg.norm(gr)
    else:
        assert abs(v - vr) <= 1e-12 * abs(vr), (v, vr)
        assert np.linalg.norm(g - gr) <= 1e-8 * np.linalg.norm(gr)


def test_streamed_fp64_matches_oracle_and_set_path():
    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    o = P.oracle_for(name)
    data = P.data_sample(name, 300_000)           # two pieces each
    norm = P.uniform_sample(name, 400_000)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    p = synth.perturbed_params(spec, 3)
    v, g = lik.nll_grad_streamed(p, torch.from_numpy(data), torch.from_numpy(norm))
    vr, gr = o.nll_grad(p, data, norm)
    check(v, g, vr, gr, False)
    # the stored samples are the inputs, and the regular call on them agrees
    np.testing.assert_array_equal(rows_sorted(lik.stored_sample("data").cpu().numpy()),
                                  rows_sorted(data))
    np.testing.assert_array_equal(rows_sorted(lik.stored_sample("norm").cpu().numpy()),
                                  rows_sorted(norm))
    v2, g2 = lik.nll_grad(p)
    check(v2, g2, v, g, False)
    # a second call with small samples (one piece each) and other parameters
    d2 = P.data_sample(name, 5000, seed=7)
    n2 = P.uniform_sample(name, 20_000, seed=8)
    p2 = synth.perturbed_params(spec, 4)
    v3, g3 = lik.nll_grad_streamed(p2, d2, n2)
    check(v3, g3, *o.nll_grad(p2, d2, n2), False)
    # either side of the two-piece threshold (2^16 events): an odd split of
    # the data into two pieces, the normalisation sample in one
    d3 = P.data_sample(name, 65_537, seed=9)
    n3 = P.uniform_sample(name, 65_535, seed=10)
    v5, g5 = lik.nll_grad_streamed(p2, d3, n3)
    check(v5, g5, *o.nll_grad(p2, d3, n3), False)
    # no data events: only the normalisation term, its gradient zero
    v4, g4 = lik.nll_grad_streamed(p2, np.zeros((0, 2)), n2)
    assert v4 == 0.0 and np.all(g4 == 0.0)


def test_streamed_fp32_matches_oracle_and_set_path():
    name = "kpipi_n40"
    spec = P.spec_by_name(name)
    data = P.data_sample(name, 1_000_000, f32=True)
    norm = P.uniform_sample(name, 1_000_000, f32=True)
    lik = Likelihood(0, F32)
    lik.set_spec(spec)
    p = synth.perturbed_params(spec, 5)
    v, g = lik.nll_grad_streamed(p, torch.from_numpy(data).pin_memory(),
                                 torch.from_numpy(norm).pin_memory())
    vr, gr = P.oracle_for(name).nll_grad(p, data.astype(np.float64), norm.astype(np.float64))
    check(v, g, vr, gr, True)
    ref = Likelihood(0, F32)
    ref.set_spec(spec)
    ref.set_events(data)
    ref.set_norm_sample(norm)
    vs, gs = ref.nll_grad(p)
    check(v, g, vs, gs, True)


def test_streamed_outside_event_keeps_state():
    name = "pipipi_n30"
    spec = P.spec_by_name(name)
    data = P.data_sample(name, 100_000)
    norm = P.uniform_sample(name, 200_000)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    p = synth.perturbed_params(spec, 6)
    v, g = lik.nll_grad_streamed(p, data, norm)
    bad = norm.copy()
    bad[150_001] = (0.01, 0.01)                      # in the second half
    with pytest.raises(MipwaError, match="EOUTSIDE") as err:
        lik.nll_grad_streamed(p, data, bad)
    assert err.value.n_outside == 1
    v2, g2 = lik.nll_grad(p)
    check(v2, g2, v, g, False)


def test_streamed_state_rules():
    name = "pipipi_n10"
    spec = P.spec_by_name(name)
    data = P.data_sample(name, 3000)
    norm = P.grid_sample(name, 60)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    p = synth.perturbed_params(spec, 2)
    lik.enable_basis_cache(True)
    with pytest.raises(MipwaError, match="ESTATE"):
        lik.nll_grad_streamed(p, data, norm)
    lik.enable_basis_cache(False)
    with pytest.raises(ValueError):
        lik.nll_grad_streamed(p, torch.from_numpy(data).cuda(), norm)
    v, g = lik.nll_grad_streamed(p, data, norm)
    check(v, g, *P.oracle_for(name).nll_grad(p, data, norm), False)


def test_streamed_then_moment_normalisation():
    """A sample grouped piece by piece is grouped as a whole before the
    per-cell moments are built (Re/Im form)."""
    name = "pipipi_n30_reim"
    spec = P.spec_by_name(name)
    data = P.data_sample(name, 50_000)
    norm = P.uniform_sample(name, 300_000)
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    p = synth.perturbed_params(spec, 9)
    v, g = lik.nll_grad_streamed(p, data, norm)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    check(v, g, vr, gr, False)
    lik.enable_norm_gram(True)
    v2, g2 = lik.nll_grad(p)
    check(v2, g2, vr, gr, False)
