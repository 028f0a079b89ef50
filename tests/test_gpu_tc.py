"""Normalisation integrals of many toys with the spline values from the tensor
cores (mipwa_toys_norm_tc): the products a_t(s), phi_t(s) of the first tile
against the FP64 natural spline of each toy's knot values (the oracle's
spline routines), and the integrals I_t = mean |A_t|^2 against the oracle's
|A|^2 summed in FP64. 200 toys (a full and a partial group of 128) and a
normalisation sample whose last tile of 64 events is ragged.

The tolerances are the FP32 form's: the spline values within 1e-6 of
max(1, |value|) (three-part bf16 operands, FP32 accumulation), the integrals
within 1e-6 relative; the measured errors are reported by the benchmark."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, Likelihood  # noqa: E402

N_TOYS = 200
N_NORM = 100_003


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.fixture(scope="module")
def problem():
    name = "pipipi_n30"
    spec = P.spec_by_name(name)
    norm = P.uniform_sample(name, N_NORM, f32=True)
    pool = P.data_sample(name, 10 * N_TOYS, seed=5, f32=True)
    offsets = np.arange(N_TOYS + 1, dtype=np.int64) * 10
    params = np.stack([synth.perturbed_params(spec, 300 + t) for t in range(N_TOYS)])
    lik = Likelihood(0, F32)
    lik.set_spec(spec)
    lik.set_norm_sample(torch.from_numpy(norm).to("cuda:0"))
    lik.set_toys(torch.from_numpy(pool).to("cuda:0"), offsets)
    lik.enable_basis_cache(True)
    stored = lik.stored_sample("norm").cpu().numpy().astype(np.float64)
    return name, spec, lik, params, stored


def test_tc_spline_values_match_fp64_spline(problem):
    name, spec, lik, params, stored = problem
    vals, ms = lik.toys_norm_tc(params, mode=1)
    assert ms > 0
    R, N = spec.n_res, spec.n_knots
    x = np.asarray(spec.knots)
    ev = stored[:64]
    worst = 0.0
    for t in range(128):
        for which in range(2):
            y = params[t, 2 * R + which * N: 2 * R + (which + 1) * N]
            M = oracle.spline_second_derivs(x, y)
            for ch in range(2):
                ref = oracle.spline_eval(x, y, M, ev[:, ch])
                got = vals[2 * ch + which, t]
                err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
                worst = max(worst, float(err.max()))
    assert worst < 1e-6, worst


def test_tc_integrals_match_oracle(problem):
    name, spec, lik, params, stored = problem
    I, ms = lik.toys_norm_tc(params, mode=0)
    o = P.oracle_for(name)
    for t in list(range(0, N_TOYS, 9)) + [N_TOYS - 1]:
        ref = float(np.mean(o.amp2(params[t], stored)))
        assert abs(I[t] - ref) <= 1e-6 * ref, (t, I[t], ref)
    # the cached basis is reused, and a new sample is picked up
    I2, _ = lik.toys_norm_tc(params, mode=0)
    np.testing.assert_allclose(I2, I, rtol=1e-12)


def test_tc_errors(problem):
    """The entry point's refusals: a bad mode or parameter, FP64 mode, and
    no toys yet."""
    import ctypes
    from paper_1703_03284_gb300 import F64, MipwaError, _lib
    name, spec, lik, params, stored = problem
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.toys_norm_tc(params, mode=2)
    bad = params.copy()
    bad[3, 0] = np.nan
    with pytest.raises(MipwaError, match="EINVAL"):
        lik.toys_norm_tc(bad, mode=0)
    norm = torch.from_numpy(P.uniform_sample(name, 1000, f32=True)).to("cuda:0")
    pool = torch.from_numpy(P.data_sample(name, 20, seed=6, f32=True)).to("cuda:0")
    l64 = Likelihood(0, F64)
    l64.set_spec(spec)
    l64.set_norm_sample(norm)
    l64.set_toys(pool, np.array([0, 10, 20], dtype=np.int64))
    with pytest.raises(MipwaError, match="ESTATE"):
        l64.toys_norm_tc(params[:2], mode=0)
    # no toys set: the C entry point itself refuses
    l32 = Likelihood(0, F32)
    l32.set_spec(spec)
    l32.set_norm_sample(norm)
    p = np.ascontiguousarray(params[0])
    out = np.zeros(1)
    ms = ctypes.c_double(0.0)
    pd = ctypes.POINTER(ctypes.c_double)
    rc = l32._lib.mipwa_toys_norm_tc(l32._h, p.ctypes.data_as(pd), 0, out.ctypes.data_as(pd),
                                     ctypes.byref(ms))
    assert rc == _lib.ESTATE
