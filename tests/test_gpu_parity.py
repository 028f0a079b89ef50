"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated for the method's accuracy targets):
  * FP64 form: NLL within 1e-12 relative, gradient within 1e-8 (norm-wise
    relative), per-event |A|^2 within 1e-12 relative;
  * FP32-mixed form: per-event |A|^2 within 1e-5 relative of the oracle fed the
    same float32-rounded (s12, s13); NLL within 1e-2 absolute at 10^7 events
    (tested here at 10^6 events with the same bound);
  * Dalitz-boundary classification: identical (an integer decision, both sides FP64).
"""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

lib_mod = pytest.importorskip("paper_1703_03284_gb300")
from paper_1703_03284_gb300 import F32, F64, Likelihood, MipwaError  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def make(name, data, norm, mode=F64):
    lik = Likelihood(0, mode)
    lik.set_spec(P.spec_by_name(name))
    lik.set_events(torch.from_numpy(np.ascontiguousarray(data)).to(DEV))
    lik.set_norm_sample(torch.from_numpy(np.ascontiguousarray(norm)).to(DEV))
    return lik


def rel(a, b):
    return abs(a - b) / abs(b)


def grad_rel(g, gref):
    return np.linalg.norm(g - gref) / np.linalg.norm(gref)


# ------------------------------------------------------------------ FP64 form
@pytest.mark.parametrize("which", ["true", "perturbed"])
def test_fp64_small_config(which):
    """10^4 accept-reject events, 10 knots, normalisation on the in-boundary
    centres of a 100 x 100 grid; FP64 throughout."""
    name = "pipipi_n10"
    data, norm = P.data_sample(name, 10_000), P.grid_sample(name, 100)
    spec = P.spec_by_name(name)
    p = synth.true_params(spec) if which == "true" else synth.perturbed_params(spec, 3)
    lik = make(name, data, norm)
    v, g = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8
    assert rel(lik.nll(p), v) < 1e-14


@pytest.mark.parametrize("name", ["pipipi_n30", "pipipi_n40", "kpipi_n40", "kkk_n40"])
def test_fp64_models(name):
    data, norm = P.data_sample(name, 20_000), P.uniform_sample(name, 30_000)
    spec = P.spec_by_name(name)
    p = synth.perturbed_params(spec, 5)
    lik = make(name, data, norm)
    v, g = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8


@pytest.mark.parametrize("nd,nn", [(1, 1), (255, 257), (257, 4097), (1023, 1), (5000, 300)])
def test_fp64_ragged_sizes(nd, nn):
    name = "pipipi_n10"
    data = P.data_sample(name, 6000)[:nd]
    norm = P.uniform_sample(name, 5000)[:nn]
    p = synth.perturbed_params(P.spec_by_name(name), 7)
    lik = make(name, data, norm)
    v, g = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8


def test_empty_data_sample():
    name = "pipipi_n10"
    norm = P.grid_sample(name, 50)
    p = synth.true_params(P.spec_by_name(name))
    lik = make(name, np.zeros((0, 2)), norm)
    v, g = lik.nll_grad(p)
    assert v == 0.0
    assert np.all(g == 0.0)


def test_fp64_amp2_per_event():
    for name in ("pipipi_n10", "kpipi_n40"):
        spec = P.spec_by_name(name)
        o = P.oracle_for(name)
        ev = P.uniform_sample(name, 50_001)
        p = synth.perturbed_params(spec, 9)
        lik = Likelihood(0, F64)
        lik.set_spec(spec)
        got = lik.amp2(p, torch.from_numpy(ev).to(DEV)).cpu().numpy()
        want = o.amp2(p, ev)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
        # outside points have no support
        box = spec.s_lo + (spec.s_hi - spec.s_lo) * np.random.default_rng(4).random((4000, 2))
        out = lik.amp2(p, torch.from_numpy(box).to(DEV)).cpu().numpy()
        np.testing.assert_allclose(out, o.density(p, box), rtol=1e-12, atol=0)


def test_inside_matches_oracle():
    for name in ("pipipi_n10", "kpipi_n40"):
        spec = P.spec_by_name(name)
        o = P.oracle_for(name)
        rng = np.random.default_rng(21)
        box = spec.s_lo - 0.05 + (spec.s_hi - spec.s_lo + 0.1) * rng.random((200_000, 2))
        lik = Likelihood(0, F64)
        lik.set_masses(spec.mD, spec.m1, spec.m2)
        got = lik.inside(torch.from_numpy(box).to(DEV)).cpu().numpy()
        np.testing.assert_array_equal(got, o.inside(box))
        got32 = lik.inside(torch.from_numpy(box.astype(np.float32)).to(DEV)).cpu().numpy()
        np.testing.assert_array_equal(got32, o.inside(box.astype(np.float32).astype(np.float64)))


def _near_boundary(spec, n, seed):
    """Points placed relative 1e-9 .. 1e-3 off the Dalitz boundary (both
    edges of the s23 range at fixed s12, and s12 near its thresholds), in
    both orders of (s12, s13)."""
    rng = np.random.default_rng(seed)
    m1, m2, mD = spec.m1, spec.m2, spec.mD
    smin, smax = (m1 + m2) ** 2, (mD - m2) ** 2
    t = np.concatenate([rng.uniform(smin, smax, n // 2),
                        smin * (1 + 10 ** rng.uniform(-7, -1, n // 4)),
                        smax * (1 - 10 ** rng.uniform(-7, -1, n - n // 2 - n // 4))])
    e2 = (t - m1 * m1 + m2 * m2) / (2 * np.sqrt(t))
    e3 = (mD * mD - t - m2 * m2) / (2 * np.sqrt(t))
    k2 = np.sqrt(np.maximum(e2 * e2 - m2 * m2, 0))
    k3 = np.sqrt(np.maximum(e3 * e3 - m2 * m2, 0))
    es = (e2 + e3) ** 2
    b = np.where(rng.random(n) < 0.5, es - (k2 + k3) ** 2, es - (k2 - k3) ** 2)
    b = b * (1 + rng.choice([-1, 1], n) * 10 ** rng.uniform(-9, -3, n))
    s13 = (mD * mD + m1 * m1 + 2 * m2 * m2) - t - b
    pts = np.stack([np.concatenate([t, s13]), np.concatenate([s13, t])], axis=1)
    return pts


def test_inside_near_boundary_matches_oracle():
    """float32 events within 1e-9 .. 1e-3 (relative) of the boundary: the FP32
    decision with its error margin, and the FP64 test behind it, classify
    exactly as the oracle does on the same float32 values."""
    for name in ("pipipi_n10", "kpipi_n40", "kkk_n40"):
        spec = P.spec_by_name(name)
        o = P.oracle_for(name)
        pts = _near_boundary(spec, 400_000, 5).astype(np.float32)
        lik = Likelihood(0, F32)
        lik.set_masses(spec.mD, spec.m1, spec.m2)
        got = lik.inside(torch.from_numpy(pts).to(DEV)).cpu().numpy()
        ref = o.inside(pts.astype(np.float64))
        assert 0.2 < ref.mean() < 0.8
        np.testing.assert_array_equal(got, ref)


def test_set_events_rejects_outside_and_keeps_state():
    name = "pipipi_n10"
    data, norm = P.data_sample(name, 3000), P.grid_sample(name, 50)
    p = synth.true_params(P.spec_by_name(name))
    lik = make(name, data, norm)
    v0 = lik.nll(p)
    bad = data.copy()
    bad[[5, 17, 2000]] = [[0.01, 0.01], [3.5, 0.5], [2.9, 2.9]]
    with pytest.raises(MipwaError) as e:
        lik.set_events(torch.from_numpy(bad).to(DEV))
    assert e.value.status == -2 and e.value.n_outside == 3
    assert lik.nll(p) == v0


def test_call_order_and_argument_errors():
    name = "pipipi_n10"
    spec = P.spec_by_name(name)
    lik = Likelihood(0, F64)
    with pytest.raises(MipwaError) as e:
        lik.set_events(np.zeros((3, 2)))
    assert e.value.status == -6
    lik.set_masses(spec.mD, spec.m1, spec.m2)
    with pytest.raises(MipwaError) as e:
        lik.set_model(spec.resonances, spec.knots[::-1], spec.r_res, spec.r_D)
    assert e.value.status == -1
    with pytest.raises(MipwaError) as e:
        lik.set_model(((0.1, 0.1, 1),), spec.knots, spec.r_res, spec.r_D)  # below threshold
    assert e.value.status == -1
    lik.set_model(spec.resonances, spec.knots, spec.r_res, spec.r_D)
    with pytest.raises(MipwaError) as e:
        lik.nll(synth.true_params(spec))
    assert e.value.status == -6
    lik.set_events(P.data_sample(name, 100))
    with pytest.raises(MipwaError) as e:
        lik.set_norm_sample(np.zeros((0, 2)))
    assert e.value.status == -1
    lik.set_norm_sample(P.grid_sample(name, 30))
    p = synth.true_params(spec)
    p[3] = np.nan
    with pytest.raises(MipwaError) as e:
        lik.nll(p)
    assert e.value.status == -1


def test_nonpositive_amplitude_is_an_error():
    name = "pipipi_n10"
    lik = make(name, P.data_sample(name, 500), P.grid_sample(name, 40))
    with pytest.raises(MipwaError) as e:
        lik.nll(np.zeros(P.spec_by_name(name).n_params))
    assert e.value.status == -3


def test_nonuniform_knots_and_spin0():
    spec = synth.ModelSpec(name="custom", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=((0.77526, 0.1491, 1), (0.98, 0.06, 0), (1.2755, 0.1867, 2)),
                           knots=(0.078, 0.2, 0.45, 0.8, 0.95, 1.3, 1.9, 2.5, 2.987))
    import oracle
    o = oracle.Oracle(spec)
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    pts = synth.uniform_in_plot(spec, 20_000, ins, seed=5).numpy()
    data, norm = pts[:8000], pts[8000:]
    rng = np.random.default_rng(2)
    p = np.concatenate([[0.2, 0.0, 0.1, 0.3, 0.3, -0.1], 1 + 0.3 * rng.random(9),
                        np.linspace(0, 2.5, 9)])
    lik = Likelihood(0, F64)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    v, g = lik.nll_grad(p)
    vr, gr = o.nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8


def test_fp64_gradient_central_differences():
    name = "kpipi_n40"
    lik = make(name, P.data_sample(name, 10_000), P.uniform_sample(name, 10_000))
    p = synth.perturbed_params(P.spec_by_name(name), 13)
    _, g = lik.nll_grad(p)
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (lik.nll(p + e) - lik.nll(p - e)) / (2 * h)
    assert grad_rel(g, fd) < 1e-6


def test_nll_is_deterministic():
    name = "pipipi_n40"
    lik = make(name, P.data_sample(name, 100_000), P.uniform_sample(name, 100_000))
    p = synth.perturbed_params(P.spec_by_name(name), 1)
    a = [lik.nll(p) for _ in range(3)]
    assert a[0] == a[1] == a[2]
    g = [lik.nll_grad(p)[1] for _ in range(2)]
    np.testing.assert_allclose(g[0], g[1], rtol=1e-13, atol=1e-13 * np.abs(g[0]).max())


def test_autograd_function_matches_gradient():
    from paper_1703_03284_gb300.autograd import MipwaNLL

    name = "pipipi_n10"
    lik = make(name, P.data_sample(name, 4000), P.grid_sample(name, 60))
    p0 = synth.perturbed_params(P.spec_by_name(name), 2)
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    y = MipwaNLL.apply(p, lik)
    (3.0 * y).backward()
    v, g = lik.nll_grad(p0)
    # forward (NLL-only kernel) and backward (NLL+gradient kernel) sum in the
    # same order; FMA contraction may still differ in the last bit
    assert abs(float(y.detach()) - v) <= 1e-14 * abs(v)
    # the gradient bins are accumulated with shared-memory atomics, whose order
    # varies between launches: equal to ~1e-13, not bitwise
    np.testing.assert_allclose(p.grad.numpy(), 3.0 * g, rtol=1e-12, atol=1e-12 * np.abs(g).max())


# ---------------------------------------------------------------- FP32 form
# Per-event |A|^2 in FP32: relative error below 1e-5 for events drawn from
# the PDF. Uniform phase-space events near a zero of A (destructive
# interference) have a relative error that grows as 1/|A|: there the bound is
# 1e-5 relative plus 1e-8 of the mean intensity in absolute terms, and at most
# 0.1% of events may exceed 1e-5 relative.
def test_fp32_amp2_per_event():
    for name in ("pipipi_n40", "kpipi_n40"):
        spec = P.spec_by_name(name)
        o = P.oracle_for(name)
        lik = Likelihood(0, F32)
        lik.set_spec(spec)
        truth = synth.true_params(spec)
        data32 = P.data_sample(name, 200_000, f32=True)
        got = lik.amp2(truth, torch.from_numpy(data32).to(DEV)).cpu().numpy()
        want = o.amp2(truth, data32.astype(np.float64))
        assert np.abs(got / want - 1).max() < 1e-5
        for p in (truth, synth.perturbed_params(spec, 9)):
            ev32 = P.uniform_sample(name, 200_000, f32=True)
            got = lik.amp2(p, torch.from_numpy(ev32).to(DEV)).cpu().numpy()
            want = o.amp2(p, ev32.astype(np.float64))
            err = np.abs(got - want)
            assert np.all(err <= 1e-5 * want + 1e-8 * want.mean())
            assert np.mean(err > 1e-5 * want) < 1e-3


def _fp32_nll_check(name, n, tol):
    data = P.data_sample(name, n, f32=True)
    norm = P.uniform_sample(name, n, f32=True)
    spec = P.spec_by_name(name)
    lik = make(name, data, norm, mode=F32)
    d64, n64 = data.astype(np.float64), norm.astype(np.float64)
    for p in (synth.true_params(spec), synth.perturbed_params(spec, 4)):
        v, g = lik.nll_grad(p)
        vr, gr = P.oracle_for(name).nll_grad(p, d64, n64)
        assert abs(v - vr) < tol, (v, vr)
        # FP32 gradient, measured at 1e7 + 1e7 events: ~5e-8 relative at the
        # perturbed point; ~1.2e-5 at the truth, near the minimum, where the
        # gradient is small and the FP32 rounding of the large per-cell adjoint
        # sums dominates (repeated calls differ by up to ~1e-5 there: the
        # shared-memory bins add in arrival order). The fit test bounds the
        # effect on the fitted parameters.
        assert grad_rel(g, gr) < 2e-5
        assert abs(lik.nll(p) - v) < 1e-3


@pytest.mark.parametrize("name", ["pipipi_n40", "kpipi_n40"])
def test_fp32_nll_1e6(name):
    _fp32_nll_check(name, 1_000_000, 1e-2)


@pytest.mark.slow
def test_fp32_nll_1e7():
    """The stated target: NLL within 1e-2 absolute at 10^7 + 10^7 events."""
    _fp32_nll_check("pipipi_n40", 10_000_000, 1e-2)


def test_model_after_samples_regroups_events():
    """set_model after the samples were stored re-groups them by spline cell;
    the result must not depend on the call order."""
    name = "kpipi_n40"
    spec = P.spec_by_name(name)
    data, norm = P.data_sample(name, 20_000), P.uniform_sample(name, 30_000)
    p = synth.perturbed_params(spec, 5)
    lik = Likelihood(0, F64)
    lik.set_masses(spec.mD, spec.m1, spec.m2)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    lik.set_model(spec.resonances, spec.knots, spec.r_res, spec.r_D)
    v, g = lik.nll_grad(p)
    vr, gr = P.oracle_for(name).nll_grad(p, data, norm)
    assert rel(v, vr) < 1e-12
    assert grad_rel(g, gr) < 1e-8
    # a different knot grid re-groups again
    knots = np.linspace(spec.knots[0], spec.knots[-1], 17)
    lik.set_model(spec.resonances, knots, spec.r_res, spec.r_D)
    spec2 = synth.ModelSpec(name="k17", mD=spec.mD, m1=spec.m1, m2=spec.m2,
                            resonances=spec.resonances, knots=tuple(knots))
    import oracle
    p2 = synth.perturbed_params(spec2, 6)
    v2, g2 = lik.nll_grad(p2)
    vr2, gr2 = oracle.Oracle(spec2).nll_grad(p2, data, norm)
    assert rel(v2, vr2) < 1e-12
    assert grad_rel(g2, gr2) < 1e-8


@pytest.mark.parametrize("mode", [F64, F32], ids=["fp64", "fp32"])
def test_basis_cache(mode):
    """With the cached Breit-Wigner basis the result matches the oracle as the
    direct form does, and the cache follows compute-mode and model changes."""
    name = "kpipi_n40"
    spec = P.spec_by_name(name)
    f32 = mode == F32
    data = P.data_sample(name, 200_000, f32=f32)
    norm = P.uniform_sample(name, 200_000, f32=f32)
    d64, n64 = data.astype(np.float64), norm.astype(np.float64)
    lik = make(name, data, norm, mode=mode)
    lik.enable_basis_cache(True)
    o = P.oracle_for(name)
    p = synth.perturbed_params(spec, 12)
    vr, gr = o.nll_grad(p, d64, n64)

    def check(v, g, m):
        if m == F32:
            assert abs(v - vr) < 1e-2 and grad_rel(g, gr) < 1e-5
        else:
            assert rel(v, vr) < 1e-12 and grad_rel(g, gr) < 1e-8

    v, g = lik.nll_grad(p)
    check(v, g, mode)
    v2, g2 = lik.nll_grad(p)  # cache reused
    check(v2, g2, mode)
    other = F64 if f32 else F32
    lik.set_compute_mode(other)
    v3, g3 = lik.nll_grad(p)
    check(v3, g3, other)
    lik.set_compute_mode(mode)
    lik.enable_basis_cache(False)
    v4, g4 = lik.nll_grad(p)
    check(v4, g4, mode)


# ------------------------------------------ FP32-mixed form on other models
def _fp32_vs_oracle(spec, o, data, norm, params_list, nll_tol=1e-2, grad_tol=2e-5):
    d32, n32 = data.astype(np.float32), norm.astype(np.float32)
    lik = Likelihood(0, F32)
    lik.set_spec(spec)
    lik.set_events(torch.from_numpy(d32).to(DEV))
    lik.set_norm_sample(torch.from_numpy(n32).to(DEV))
    for p in params_list:
        v, g = lik.nll_grad(p)
        vr, gr = o.nll_grad(p, d32.astype(np.float64), n32.astype(np.float64))
        assert abs(v - vr) < nll_tol, (v, vr)
        assert grad_rel(g, gr) < grad_tol


def test_fp32_narrow_phi_kkk():
    """K K K with the narrow phi(1020) (4 MeV): the FP32 form keeps m_r^2 - s
    exact near the pole, so the NLL stays within tolerance at 10^6 events."""
    name = "kkk_n40"
    spec = P.spec_by_name(name)
    data = P.data_sample(name, 1_000_000, f32=True)
    norm = P.uniform_sample(name, 1_000_000, f32=True)
    # a sizeable share of the events sits within a few widths of the pole
    near = np.abs(np.minimum(data[:, 0], data[:, 1]) - 1.019461 ** 2) < 0.02
    assert near.mean() > 0.05
    _fp32_vs_oracle(spec, P.oracle_for(name), data, norm,
                    [synth.true_params(spec), synth.perturbed_params(spec, 8, 0.02)])


def test_fp32_nonuniform_knots_three_resonances():
    """Non-uniform knots (segment search instead of the uniform index) and three
    resonances including a scalar one: the generic FP32 kernel."""
    spec = synth.ModelSpec(name="custom32", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=((0.77526, 0.1491, 1), (0.98, 0.06, 0), (1.2755, 0.1867, 2)),
                           knots=(0.078, 0.2, 0.45, 0.8, 0.95, 1.3, 1.9, 2.5, 2.987))
    import oracle
    o = oracle.Oracle(spec)
    rng = np.random.default_rng(2)
    truth = np.concatenate([[0.2, 0.0, 0.1, 0.3, 0.3, -0.1], 1 + 0.3 * rng.random(9),
                            np.linspace(0, 2.5, 9)])
    dens = synth.numpy_density(lambda x: o.density(truth, x))
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    data = synth.accept_reject(spec, 300_000, dens, seed=6, dtype=torch.float32).numpy()
    norm = synth.uniform_in_plot(spec, 300_000, ins, seed=7, dtype=torch.float32).numpy()
    p2 = truth + 0.02 * np.random.default_rng(3).standard_normal(truth.shape)
    _fp32_vs_oracle(spec, o, data.astype(np.float64), norm.astype(np.float64), [truth, p2])


def test_fp32_large_phase_steps_take_the_full_sincos():
    """Knot phases that jump by 2.5 rad between neighbours: on those segments
    the phase moves too far from its reference for the short series and the
    kernel takes the full range reduction; a mixed parameter point exercises
    both paths in one evaluation (and in one warp at segment boundaries).
    Per-event |A|^2 is held to 1e-5 relative away from zeros of A and the NLL
    to 1e-2; the gradient to 1e-3 only: these points put many events next to
    zeros of A, whose 1/|A|^2 weights magnify the FP32 error of A."""
    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    o = P.oracle_for(name)
    data = P.data_sample(name, 1_000_000, f32=True)
    norm = P.uniform_sample(name, 1_000_000, f32=True)
    R, N = spec.n_res, spec.n_knots
    truth = synth.true_params(spec)
    zig = truth.copy()
    zig[2 * R + N:] = 2.5 * (np.arange(N) % 2)
    mixed = truth.copy()
    mixed[2 * R + N + N // 2:] = truth[2 * R + N + N // 2:] + 2.5 * (np.arange(N - N // 2) % 2)
    lik = Likelihood(0, F32)
    lik.set_spec(spec)
    ev = torch.from_numpy(data[:200_000]).to(DEV)
    for p in (zig, mixed):
        got = lik.amp2(p, ev).cpu().numpy()
        want = o.amp2(p, data[:200_000].astype(np.float64))
        away = want > 1e-3 * want.mean()
        assert np.abs(got[away] / want[away] - 1).max() < 1e-5
    _fp32_vs_oracle(spec, o, data.astype(np.float64), norm.astype(np.float64), [zig, mixed],
                    grad_tol=1e-3)
