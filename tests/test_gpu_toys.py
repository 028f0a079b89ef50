"""Batched toys (one launch for many toy samples sharing a normalisation
sample) against the oracle, toy by toy.

Two problem sizes: a small one where every toy is one work item, and a
work-list one whose normalisation sample spans several chunks (400,000 events
at 131,072 per item: three full chunks and a ragged fourth) and whose toys
span up to three data items (150,000 events at 65,536), so that toys own
several rows, items come chunk-major and the per-toy reduction sums several
normalisation rows, as in the 256-toy benchmark configuration."""
import functools
import itertools

import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, F64, Likelihood  # noqa: E402

SIZES = [0, 1, 300, 5000, 257, 20000]
# work-list sizes: empty, one event, a ragged block, two and three data
# items, then 16 toys of 1e3..1e5 events (Poisson around log-uniform means)
WL_SIZES = [0, 1, 257, 70_000, 150_000] + [int(x) for x in
                                           synth.toy_sizes(16, seed=9, lo_exp=3.0, hi_exp=5.0)]
WL_NORM = 400_000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def toy_problem(name, f32, sizes=SIZES, n_norm=40_000):
    spec = P.spec_by_name(name)
    pool = P.data_sample(name, sum(sizes), seed=5, f32=f32)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    norm = P.uniform_sample(name, n_norm, f32=f32)
    params = np.stack([synth.perturbed_params(spec, 100 + t) for t in range(len(sizes))])
    return spec, pool, offsets, norm, params


@functools.lru_cache(maxsize=None)
def oracle_toys(name, f32, sizes, n_norm):
    """(nll, grad) of every toy from the oracle (FP64, the same float values)."""
    spec, pool, offsets, norm, params = toy_problem(name, f32, list(sizes), n_norm)
    o = P.oracle_for(name)
    out = []
    for t in range(len(sizes)):
        d = pool[offsets[t]:offsets[t + 1]].astype(np.float64)
        out.append(o.nll_grad(params[t], d, norm.astype(np.float64)))
    return out


def make_toys(name, pool, offsets, norm, mode, cached=False, graph=True):
    lik = Likelihood(0, mode)
    lik.set_spec(P.spec_by_name(name))
    lik.set_norm_sample(torch.from_numpy(norm).to("cuda:0"))
    lik.set_toys(torch.from_numpy(pool).to("cuda:0"), offsets)
    lik.enable_basis_cache(cached)
    lik.set_toys_graph(graph)
    return lik


def check_toys(nll, grad, ref, sizes, f32):
    for t in range(len(sizes)):
        vr, gr = ref[t]
        if f32:
            assert abs(nll[t] - vr) < 1e-2, (t, nll[t], vr)
        else:
            assert abs(nll[t] - vr) <= 1e-12 * max(abs(vr), 1.0), (t, nll[t], vr)
        if sizes[t] == 0:
            assert np.all(grad[t] == 0.0), t
        else:
            err = np.linalg.norm(grad[t] - gr) / np.linalg.norm(gr)
            assert err <= (1e-5 if f32 else 1e-8), (t, err)


@pytest.mark.parametrize("cached", [False, True], ids=["direct", "cached"])
@pytest.mark.parametrize("graph", [True, False], ids=["graph", "nograph"])
def test_toys_fp64_match_oracle(cached, graph):
    name = "pipipi_n30"
    spec, pool, offsets, norm, params = toy_problem(name, False)
    lik = make_toys(name, pool, offsets, norm, F64, cached, graph)
    nll, grad = lik.nll_grad_toys(params)
    check_toys(nll, grad, oracle_toys(name, False, tuple(SIZES), 40_000), SIZES, False)
    # repeat: the work queue and the flags are reset by the launch itself
    nll2, grad2 = lik.nll_grad_toys(params)
    np.testing.assert_allclose(nll2, nll, rtol=1e-14, atol=1e-9)


@pytest.mark.parametrize("cached", [False, True], ids=["direct", "cached"])
@pytest.mark.parametrize("graph", [True, False], ids=["graph", "nograph"])
def test_toys_worklist_fp64_match_oracle(cached, graph):
    """Several normalisation chunks (the last ragged) and up to three data
    items per toy: rows t*rpt + ch and t*rpt + C + d, chunk-major items, and
    the reduction over several normalisation rows, FP64 against the oracle."""
    name = "pipipi_n30"
    spec, pool, offsets, norm, params = toy_problem(name, False, WL_SIZES, WL_NORM)
    lik = make_toys(name, pool, offsets, norm, F64, cached, graph)
    lik.set_toys_config(norm_chunk=131072, data_chunk=65536)
    nll, grad = lik.nll_grad_toys(params)
    check_toys(nll, grad, oracle_toys(name, False, tuple(WL_SIZES), WL_NORM), WL_SIZES, False)
    nll2, _ = lik.nll_grad_toys(params)
    np.testing.assert_allclose(nll2, nll, rtol=1e-14, atol=1e-9)


@pytest.mark.parametrize("cached", [False, True], ids=["direct", "cached"])
def test_toys_worklist_fp32_match_oracle(cached):
    name = "kpipi_n40"
    spec, pool, offsets, norm, params = toy_problem(name, True, WL_SIZES, WL_NORM)
    lik = make_toys(name, pool, offsets, norm, F32, cached)
    lik.set_toys_config(norm_chunk=131072, data_chunk=65536)
    nll, grad = lik.nll_grad_toys(params)
    check_toys(nll, grad, oracle_toys(name, True, tuple(WL_SIZES), WL_NORM), WL_SIZES, True)


def test_toys_worklist_every_launch_configuration():
    """Every value of every autotuner knob (normalisation chunk, data chunk,
    block size, blocks per SM) gives the oracle's result to the FP64 bar."""
    name = "pipipi_n30"
    spec, pool, offsets, norm, params = toy_problem(name, False, WL_SIZES, WL_NORM)
    ref = oracle_toys(name, False, tuple(WL_SIZES), WL_NORM)
    lik = make_toys(name, pool, offsets, norm, F64, cached=True)
    for nc, dc, bs, bps in itertools.product((65536, 131072, 262144, 524288),
                                             (32768, 65536, 131072, 262144),
                                             (128, 256, 512), (1, 0)):
        lik.set_toys_config(norm_chunk=nc, data_chunk=dc, block=bs, blocks_per_sm=bps)
        nll, grad = lik.nll_grad_toys(params)
        check_toys(nll, grad, ref, WL_SIZES, False)


def test_toys_fp32_autotune_and_cache(tmp_path):
    """The autotuner times several configurations on a sample where its
    candidates differ in chunk counts, keeps one at which the results still
    match the oracle, and reuses its choice without timing: from the context,
    and in a new context from the tune file."""
    name = "kpipi_n40"
    spec, pool, offsets, norm, params = toy_problem(name, True, WL_SIZES, WL_NORM)
    ref = oracle_toys(name, True, tuple(WL_SIZES), WL_NORM)
    lik = make_toys(name, pool, offsets, norm, F32, cached=True)
    tune = tmp_path / "toys.tune"
    lik.set_toys_tune_file(str(tune))
    best = lik.toys_autotune(params)
    assert best["n_timed"] >= 8, best
    assert best["norm_chunk"] in (65536, 131072, 262144, 524288, 1048576, 2097152)
    assert best["block"] in (128, 256, 512)
    cfg = lik.toys_config()
    assert {k: cfg[k] for k in cfg} == {k: best[k] for k in cfg}
    nll, grad = lik.nll_grad_toys(params)
    check_toys(nll, grad, ref, WL_SIZES, True)
    again = lik.toys_autotune(params)
    assert again["n_timed"] == 0 and {k: again[k] for k in cfg} == {k: best[k] for k in cfg}
    assert tune.read_text().count("\n") == 1
    other = make_toys(name, pool, offsets, norm, F32, cached=True)
    other.set_toys_tune_file(str(tune))
    from_file = other.toys_autotune(params)
    assert from_file["n_timed"] == 0 and {k: from_file[k] for k in cfg} == {k: best[k] for k in cfg}
    # another sample size is another key: timed again
    other.set_toys(torch.from_numpy(pool[:offsets[5]]).to("cuda:0"), offsets[:6])
    assert other.toys_autotune(params[:5])["n_timed"] > 0


def test_toys_fp32_match_oracle():
    name = "kpipi_n40"
    spec, pool, offsets, norm, params = toy_problem(name, True)
    lik = make_toys(name, pool, offsets, norm, F32, cached=True)
    nll, grad = lik.nll_grad_toys(params)
    check_toys(nll, grad, oracle_toys(name, True, tuple(SIZES), 40_000), SIZES, True)


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


def test_toys_config_refusals():
    """Out-of-range launch configurations are refused and leave the current
    one in place."""
    from paper_1703_03284_gb300 import MipwaError
    name = "kpipi_n40"
    spec, pool, offsets, norm, params = toy_problem(name, True)
    lik = make_toys(name, pool, offsets, norm, F32, cached=True)
    lik.set_toys_config(norm_chunk=131072, data_chunk=65536, block=256, blocks_per_sm=2)
    before = lik.toys_config()
    for bad in (dict(norm_chunk=100), dict(data_chunk=(1 << 30) + 1), dict(block=100),
                dict(block=1024), dict(blocks_per_sm=17), dict(blocks_per_sm=-1)):
        with pytest.raises(MipwaError, match="EINVAL"):
            lik.set_toys_config(**bad)
        assert lik.toys_config() == before
    nll, grad = lik.nll_grad_toys(params)
    check_toys(nll, grad, oracle_toys(name, True, tuple(SIZES), 40_000), SIZES, True)


@pytest.mark.parametrize("mode", [F64, F32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("cached", [False, True], ids=["direct", "cached"])
def test_nll_toys_without_gradient(mode, cached):
    """mipwa_nll_toys (no adjoint work) on the work-list problem: every toy's
    -2 ln L against the oracle (FP64 1e-12 relative, FP32 1e-2 absolute) and
    against mipwa_nll_grad_toys, alternating the two calls (the captured graph
    follows the mode)."""
    f32 = mode == F32
    name = "pipipi_n30" if not f32 else "kpipi_n40"
    spec, pool, offsets, norm, params = toy_problem(name, f32, WL_SIZES, WL_NORM)
    ref = oracle_toys(name, f32, tuple(WL_SIZES), WL_NORM)
    lik = make_toys(name, pool, offsets, norm, mode, cached)
    lik.set_toys_config(norm_chunk=131072, data_chunk=65536)
    nll = lik.nll_toys(params)
    for t in range(len(WL_SIZES)):
        vr = ref[t][0]
        if f32:
            assert abs(nll[t] - vr) < 1e-2, (t, nll[t], vr)
        else:
            assert abs(nll[t] - vr) <= 1e-12 * max(abs(vr), 1.0), (t, nll[t], vr)
    nll_g, grad = lik.nll_grad_toys(params)
    # the same events summed in the same order; FP32: up to FP32 rounding
    np.testing.assert_allclose(nll_g, nll, rtol=1e-12 if not f32 else 1e-7,
                               atol=1e-9 if not f32 else 1e-3)
    check_toys(nll_g, grad, ref, WL_SIZES, f32)
    np.testing.assert_array_equal(lik.nll_toys(params), nll)
