"""The batched-toy workload at full size, in the launch configuration the
benchmark times: 256 toys of the 30-knot pi pi pi model (sizes Poisson
around log-uniform means in [1e4, 1e6], about 5.5 x 10^7 events), one shared
10^7-event normalisation sample, float32 events, FP32-mixed with the cached
Breit-Wigner basis, the autotuned work list, one CUDA graph per evaluation.

Inputs come from the oracle's density and boundary only (the toys' events are
a 10^7 accept-reject sample repeated to the total; repeated events are valid
events). The oracle evaluates sampled toys one by one in FP64: the first two,
the middle one, the last one and the largest one. Tolerances are the FP32
form's: -2 ln L within 1e-2 absolute, the gradient within 1e-5 norm-wise.
Every toy: finite results, and the call without the gradient agreeing with
the one with it.
"""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, Likelihood  # noqa: E402

N_TOYS = 256
N_NORM = 10_000_000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def test_full_size_toys_vs_oracle():
    name = "pipipi_n30"
    spec = P.spec_by_name(name)
    o = P.oracle_for(name)
    sizes = synth.toy_sizes(N_TOYS, seed=7)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pool = np.resize(P.data_sample(name, 10_000_000, seed=41, f32=True), (int(offsets[-1]), 2))
    norm = synth.uniform_in_plot(
        spec, N_NORM, synth.numpy_density(lambda x: o.inside(x).astype(np.float64)),
        seed=42, dtype=torch.float32).numpy()
    params = np.stack([synth.perturbed_params(spec, 500 + t, 0.02) for t in range(N_TOYS)])
    lik = Likelihood(0, F32)
    lik.set_spec(spec)
    lik.set_norm_sample(torch.from_numpy(norm).to("cuda:0"))
    lik.set_toys(torch.from_numpy(pool).to("cuda:0"), offsets)
    lik.enable_basis_cache(True)
    best = lik.toys_autotune(params)
    assert best["n_timed"] > 0
    nll, grad = lik.nll_grad_toys(params)
    assert np.all(np.isfinite(nll)) and np.all(np.isfinite(grad))
    nll_f = lik.nll_toys(params)
    np.testing.assert_allclose(nll_f, nll, rtol=1e-7, atol=1e-3)
    norm64 = norm.astype(np.float64)
    for t in sorted({0, 1, N_TOYS // 2, N_TOYS - 1, int(np.argmax(sizes))}):
        d = pool[offsets[t]:offsets[t + 1]].astype(np.float64)
        vr, gr = o.nll_grad(params[t], d, norm64)
        assert abs(nll[t] - vr) < 1e-2, (t, nll[t], vr)
        err = np.linalg.norm(grad[t] - gr) / np.linalg.norm(gr)
        assert err <= 1e-5, (t, err)
