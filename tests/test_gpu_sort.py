"""The set-time grouping of stored samples by spline cell.

-2 ln L is a sum over events, so the library stores each sample grouped by
the pair of S-wave segments (Sec. 2) its event falls in, which lets the event
kernels read one cell's spline coefficients per warp. The stored order must be
exactly the stable sort by the key j12 (N-1) + j13, whichever path stored the
sample (a host copy counted piece by piece as it lands, a device copy, or a
re-grouping after set_model). The expected order here comes from numpy's
stable argsort of keys found by searchsorted on the knots; events closer to a
knot than 1e-4 of a segment are left out, so that no key depends on rounding.
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


def segments(knots, s):
    """Largest j in [0, N-2] with knot_j <= s (the end segments extend outward)."""
    j = np.searchsorted(knots, s, side="right") - 1
    return np.clip(j, 0, len(knots) - 2)


def away_from_knots(knots, ev):
    knots = np.asarray(knots)
    margin = 1e-4 * np.diff(knots).min()
    keep = np.ones(len(ev), bool)
    for col in (0, 1):
        s = ev[:, col].astype(np.float64)
        i = np.clip(np.searchsorted(knots, s), 1, len(knots) - 1)
        d = np.minimum(np.abs(s - knots[i - 1]), np.abs(s - knots[i]))
        keep &= d > margin
    return np.ascontiguousarray(ev[keep])


def expected_order(knots, ev):
    knots = np.asarray(knots)
    e = ev.astype(np.float64)
    key = segments(knots, e[:, 0]) * (len(knots) - 1) + segments(knots, e[:, 1])
    return np.argsort(key, kind="stable")


def nonuniform_knots(spec):
    k = spec.knots
    return tuple(np.concatenate([np.linspace(k[0], 1.0, 9), np.linspace(1.15, k[-1], 14)]))


def check_stored(lik, which, knots, ev):
    """ev: the sample in the order it was in before the grouping."""
    got = lik.stored_sample(which).cpu().numpy()
    assert got.dtype == ev.dtype and got.shape == ev.shape
    np.testing.assert_array_equal(got, ev[expected_order(knots, ev)])
    return got


@pytest.mark.parametrize("path", ["host", "device", "set_model"])
@pytest.mark.parametrize("f32", [True, False], ids=["f32", "f64"])
@pytest.mark.parametrize("n", [2, 33, 4863, 12_347, 1_000_003])
def test_stored_order_is_the_stable_cell_sort(n, f32, path):
    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    data = away_from_knots(spec.knots, P.data_sample(name, n + n // 50 + 64, f32=f32))[:n]
    norm = away_from_knots(spec.knots, P.uniform_sample(name, n + n // 50 + 64, f32=f32))[:n]
    lik = Likelihood(0, F32 if f32 else F64)
    if path == "set_model":
        lik.set_masses(spec.mD, spec.m1, spec.m2)
    else:
        lik.set_spec(spec)
    put = (lambda x: torch.from_numpy(x).to(DEV)) if path == "device" else torch.from_numpy
    lik.set_events(put(data))
    lik.set_norm_sample(put(norm))
    if path == "set_model":
        # the samples were stored before any model: kept in the order given,
        # then grouped by set_model
        np.testing.assert_array_equal(lik.stored_sample("data").cpu().numpy(), data)
        lik.set_model(spec.resonances, spec.knots, spec.r_res, spec.r_D)
    check_stored(lik, "data", spec.knots, data)
    check_stored(lik, "norm", spec.knots, norm)


@pytest.mark.parametrize("f32", [True, False], ids=["f32", "f64"])
def test_nonuniform_knots_and_regrouping(f32):
    """Knots that are not evenly spaced take the binary search; a new knot
    grid re-groups the stored samples (stably, from their stored order), and
    so does the old grid again."""
    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    knots2 = nonuniform_knots(spec)
    data = P.data_sample(name, 300_000, seed=11, f32=f32)
    norm = P.uniform_sample(name, 300_000, seed=12, f32=f32)
    data = away_from_knots(knots2, away_from_knots(spec.knots, data))
    norm = away_from_knots(knots2, away_from_knots(spec.knots, norm))
    lik = Likelihood(0, F32 if f32 else F64)
    lik.set_spec(spec)
    lik.set_events(torch.from_numpy(data))
    lik.set_norm_sample(torch.from_numpy(norm))
    d1 = check_stored(lik, "data", spec.knots, data)
    n1 = check_stored(lik, "norm", spec.knots, norm)
    lik.set_model(spec.resonances, knots2, spec.r_res, spec.r_D)
    check_stored(lik, "data", knots2, d1)
    n2 = check_stored(lik, "norm", knots2, n1)
    lik.set_model(spec.resonances, spec.knots, spec.r_res, spec.r_D)
    check_stored(lik, "norm", spec.knots, n2)


def test_events_on_the_knots_stay_a_permutation():
    """Events exactly on knots, past the end knots and repeated: whatever the
    segment decision at a tie, the stored sample is a permutation of the
    input whose keys never decrease by more than one segment."""
    name = "pipipi_n10"
    spec = P.spec_by_name(name)
    knots = np.asarray(spec.knots)
    ev = P.uniform_sample(name, 50_000, seed=3)
    ev = np.concatenate([ev, np.repeat(ev[:100], 5, axis=0)])
    o = P.oracle_for(name)
    on = np.stack(np.meshgrid(knots, knots), -1).reshape(-1, 2)
    on = on[o.inside(on).astype(bool)]
    ev = np.ascontiguousarray(np.concatenate([ev, on]))
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(torch.from_numpy(ev))
    got = lik.stored_sample("data").cpu().numpy()
    lex = lambda a: a[np.lexsort((a[:, 1], a[:, 0]))]
    np.testing.assert_array_equal(lex(got), lex(ev))
    key = segments(knots, got[:, 0]) * (len(knots) - 1) + segments(knots, got[:, 1])
    assert np.all(np.diff(key) >= -(len(knots) - 1) - 1)


def test_stored_sample_states():
    spec = P.spec_by_name("pipipi_n10")
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    with pytest.raises(MipwaError, match="ESTATE"):
        lik.stored_sample("norm")
    lik.set_events(torch.zeros((0, 2), dtype=torch.float64))
    assert lik.stored_sample("data").shape == (0, 2)
    one = P.uniform_sample("pipipi_n10", 1)
    lik.set_norm_sample(torch.from_numpy(one))
    np.testing.assert_array_equal(lik.stored_sample("norm").cpu().numpy(), one)
    with pytest.raises(KeyError):
        lik.stored_sample("toys")
