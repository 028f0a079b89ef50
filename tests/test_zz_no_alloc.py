"""The allocation-free entry point (mipwa_nll_grad_noalloc) against the
context entry point (mipwa_nll_grad), through the C ABI.

mipwa_nll_grad_noalloc is for callers that cannot allocate device memory (a
framework that owns the device heap, a serving process sized at start-up, a
plug-in whose host forbids allocation): it keeps its intermediates in one fixed
device array inside the library. Two calls in a row must both agree with the
context API within the tolerances of the parity tests (FP64: NLL 1e-12
relative, gradient 1e-8; FP32: NLL 1e-2 absolute, gradient 1e-5, 2e-5 at four
resonances as in the limits tests), which also shows that the shared array is
reset between calls. Cases: the 40-knot pi pi pi model in both modes, the
largest model the array holds (64 non-uniform knots, 4 resonances), events
stored in the other precision than the arithmetic, and the rejected calls
(sizes past the limits, host or foreign buffers, an event outside the plot).
This file is collected last so that a failure here comes after every other
test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

# rho(770) P, f0(980) S, f2(1270) D, rho(1450) P
RES4 = ((0.77526, 0.1491, 1), (0.98, 0.06, 0), (1.2755, 0.1867, 2), (1.465, 0.4, 1))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def compare(spec, data, norm, mode, seeds=(3, 4), g_tol32=1e-5):
    """Two noalloc calls in a row, each against the context entry point."""
    from paper_1703_03284_gb300 import F32, Likelihood
    from paper_1703_03284_gb300.api import nll_grad_noalloc

    lik = Likelihood(0, mode)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    for seed in seeds:
        p = synth.perturbed_params(spec, seed, 0.02)
        v_ref, g_ref = lik.nll_grad(p)
        v, g = nll_grad_noalloc(spec, p, data, norm, compute_mode=mode)
        gerr = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
        if mode == F32:
            assert abs(v - v_ref) < 1e-2, (seed, v, v_ref)
            assert gerr < g_tol32, (seed, gerr)
        else:
            assert abs(v - v_ref) <= 1e-12 * abs(v_ref), (seed, v, v_ref)
            assert gerr < 1e-8, (seed, gerr)


@pytest.mark.parametrize("mode,f32", [(0, False), (1, True)], ids=["fp64", "fp32"])
def test_noalloc_matches_context_entry_point(mode, f32):
    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    data = torch.from_numpy(P.data_sample(name, 50_000, f32=f32)).to("cuda:0")
    norm = torch.from_numpy(P.uniform_sample(name, 60_000, f32=f32)).to("cuda:0")
    compare(spec, data, norm, mode)


@pytest.mark.parametrize("mode,f32", [(0, True), (1, False)], ids=["fp64-f32events",
                                                                  "fp32-f64events"])
def test_noalloc_events_in_the_other_precision(mode, f32):
    name = "kpipi_n40"
    spec = P.spec_by_name(name)
    data = torch.from_numpy(P.data_sample(name, 40_000, f32=f32)).to("cuda:0")
    norm = torch.from_numpy(P.uniform_sample(name, 50_000, f32=f32)).to("cuda:0")
    compare(spec, data, norm, mode)


def largest_spec():
    """64 knots spaced non-uniformly (denser at low mass) and 4 resonances:
    every region of the fixed array at its largest."""
    u = np.linspace(0.0, 1.0, 64) ** 1.4
    knots = tuple(float(x) for x in 0.078 + (2.987 - 0.078) * u)
    return synth.ModelSpec(name="noalloc_n64_r4", mD=synth.M_D, m1=synth.M_PI, m2=synth.M_PI,
                           resonances=RES4, knots=knots)


@pytest.mark.parametrize("mode,f32", [(0, False), (1, True)], ids=["fp64", "fp32"])
def test_noalloc_largest_model(mode, f32):
    spec = largest_spec()
    o = oracle.Oracle(spec)
    truth = synth.true_params(spec)
    dt = torch.float32 if f32 else torch.float64
    data = synth.accept_reject(spec, 100_000, synth.numpy_density(lambda x: o.density(truth, x)),
                               seed=31, dtype=dt).to("cuda:0")
    norm = synth.uniform_in_plot(spec, 100_000, synth.numpy_density(
        lambda x: o.inside(x).astype(np.float64)), seed=32, dtype=dt).to("cuda:0")
    compare(spec, data, norm, mode, g_tol32=2e-5)


def raw_call(spec, data, norm, n_knots=None, n_res=None, d_out=None, device=0):
    """mipwa_nll_grad_noalloc with arguments that the Python wrapper would
    refuse; returns the status."""
    from paper_1703_03284_gb300 import _lib
    lib = _lib.load()
    res_list = list(spec.resonances)
    knots_list = list(spec.knots)
    R = len(res_list) if n_res is None else n_res
    N = len(knots_list) if n_knots is None else n_knots
    while len(res_list) < R:
        res_list.append((1.5, 0.1, 0))
    while len(knots_list) < N:
        knots_list.append(knots_list[-1] + 0.01)
    res = (_lib.Resonance * max(R, 1))()
    for i in range(R):
        m, w, L = res_list[i]
        res[i] = _lib.Resonance(float(m), float(w), int(L))
    knots = np.ascontiguousarray(knots_list[:N], dtype=np.float64)
    params = np.ones(2 * R + 2 * N, dtype=np.float64)
    if d_out is None:
        d_out = torch.empty(1 + len(params), dtype=torch.float64, device="cuda:0")
    code = 1 if data.dtype == torch.float32 else 0
    pd = ctypes.POINTER(ctypes.c_double)
    return lib.mipwa_nll_grad_noalloc(
        device, 0, float(spec.mD), float(spec.m1), float(spec.m2), res, R,
        knots.ctypes.data_as(pd), N, float(spec.r_res), float(spec.r_D),
        ctypes.c_void_p(data.data_ptr()), data.shape[0], ctypes.c_void_p(norm.data_ptr()),
        norm.shape[0], code, params.ctypes.data_as(pd), ctypes.c_void_p(d_out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream(0).cuda_stream))


def test_noalloc_rejected_calls():
    from paper_1703_03284_gb300 import _lib
    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    data = torch.from_numpy(P.data_sample(name, 5_000)).to("cuda:0")
    norm = torch.from_numpy(P.uniform_sample(name, 5_000)).to("cuda:0")
    assert raw_call(spec, data, norm) == _lib.OK
    # one past each limit of the fixed array: 65 knots, 5 resonances
    assert raw_call(spec, data, norm, n_knots=65) == _lib.EINVAL
    assert raw_call(spec, data, norm, n_res=5) == _lib.EINVAL
    # a host buffer where the kernels need device memory
    assert raw_call(spec, data, norm.cpu()) == _lib.EINVAL
    assert raw_call(spec, data, norm, d_out=torch.empty(200, dtype=torch.float64)) == _lib.EINVAL
    # a device index the process does not have
    assert raw_call(spec, data, norm, device=torch.cuda.device_count()) != _lib.OK
    # one normalisation event outside the Dalitz plot
    bad = norm.clone()
    bad[17] = torch.tensor([0.01, 0.01], dtype=bad.dtype)
    assert raw_call(spec, data, bad) == _lib.EOUTSIDE
    # the array was not left in a bad state: a good call still agrees
    compare(spec, data, norm, 0, seeds=(5,))
